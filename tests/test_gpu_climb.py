"""GPU parity of the Raibert-feedback gait reference (Sec. IV-B) and of the
climbing task's ground-relative height cost (Sec. IV-C) against the FP64
oracle, through the C ABI; and the closed-loop climb onto a box."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import _mppi, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_and_oracle_costs(cfg, K, H, t0, x0=None):
    m = dict(cfg.mppi, K=K, H=H)
    ctl = _mppi.Controller(cfg.robot, cfg.cost, m)
    ctl.set_nominal(cfg.mu0)
    U = torch.empty((K, 48), device="cuda")
    ctl.sample(0, out=U)
    L = torch.empty(K, device="cuda")
    x0 = (cfg.x0 if x0 is None else x0).astype(np.float32)
    ctl.rollouts(dev(x0), U=U, n=K, t0=t0, L_out=L)
    world = O.World(cfg.robot)
    Uh = U.cpu().numpy()
    Lo = O.rollouts(world, cfg.cost, m, t0, x0.astype(np.float64), Uh)
    return L.cpu().numpy().astype(np.float64), Lo, (world, m, Uh, x0.astype(np.float64))


def test_raibert_trot_cost_parity():
    cfg = W.config_trot_raibert()
    Lg, Lo, _ = gpu_and_oracle_costs(cfg, 96, 80, 0.21)
    rel = np.abs(Lg - Lo) / np.maximum(np.abs(Lo), 1.0)
    assert np.all(np.isfinite(Lg)) and rel.max() <= 1e-3, rel.max()
    # the feedback matters: the same samples under the open-loop trot cost differently
    c1 = dict(cfg.cost, gait=1)
    Lg1, _, _ = gpu_and_oracle_costs(W.Workload(cfg.name, cfg.robot, c1, cfg.mppi, cfg.x0, cfg.mu0, cfg.steps),
                                     96, 80, 0.21)
    assert np.abs(Lg1 - Lg).max() > 1.0


@pytest.mark.parametrize("start_x", [0.0, 0.9])
def test_climb_cost_parity(start_x):
    """plane + static box (the general terrain path) with the ground-relative
    height: from the start, and from a state standing on the box"""
    cfg = W.config_climb()
    x0 = cfg.x0.copy()
    if start_x > 0:
        x0[0] = start_x
        x0[2] += 0.24
    Lg, Lo, (world, m, Uh, x0d) = gpu_and_oracle_costs(cfg, 96, 60, 0.0, x0)
    rel = np.abs(Lg - Lo) / np.maximum(np.abs(Lo), 1.0)
    assert np.all(np.isfinite(Lg))
    # a box edge is a normal jump: bound each sample by max(1e-3, 3x its own FP64 sensitivity)
    sens = np.zeros_like(Lo)
    for sd in range(2):
        xp = x0d * (1 + 1e-7 * np.random.default_rng(sd).standard_normal(x0d.shape))
        Lp = O.rollouts(world, cfg.cost, m, 0.0, xp, Uh)
        sens = np.maximum(sens, np.abs(Lp - Lo) / np.maximum(np.abs(Lo), 1.0))
    assert np.percentile(rel, 95) <= 1e-3
    assert np.all(rel <= np.maximum(1e-3, 3 * sens)), (rel.max(), sens[rel.argmax()])


def test_closed_loop_climb_onto_a_box():
    """Sec. IV-C: the trot reference and a waypoint on top of a 0.24 m box
    (about the standing height); closed-loop episodes of 4 s on the GPU path
    (8 paired starts, K = 1024, H = 100).  A climb counts when the trunk is at
    least 0.15 m above the box top over its footprint, at x >= 0.75 m."""
    from paper_2409_10469_gb300 import proposal as P

    def make(e):
        return W.config_climb(K=1024, H=100, box_height=0.24)
    st, ct, cfgs = P.run_episodes(make, 8, 1024, 100, 400, seed=1)
    assert np.all(np.isfinite(st))
    x, z = st[:, :, 0], st[:, :, 2]
    climbed = np.any((x >= 0.75) & (x <= 1.65) & (z >= 0.24 + 0.15), axis=0)
    print("climbed", int(climbed.sum()), "of 8; final x", np.round(x[-1], 2).tolist())
    assert climbed.sum() >= 3
