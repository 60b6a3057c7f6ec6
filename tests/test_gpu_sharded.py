"""The K-sharded control step through the C ABI (mppi_step_partial /
mppi_step_finalize) on one GPU: `world` handles stand for the ranks, each
rolling out its own range of the step's samples; the two collectives of the
protocol run in-process.  Every rank's samples are the oracle's Philox knots at
their global indices, every rank ends with the same mean, and that mean equals
the one-kernel step over all K samples and the oracle's Eq. 1 / Eq. 2 on the
same knots and costs (<= 1e-6), step after step."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import _mppi, sharded as SH, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


@pytest.mark.parametrize("which,K,H,world", [("trot", 1000, 40, 2), ("trot", 1000, 40, 3), ("stand", 64, 30, 4),
                                             ("push", 300, 30, 2)])
def test_sharded_step_equals_the_one_kernel_step(which, K, H, world):
    cfg = {"trot": W.config_trot, "stand": W.config_stand, "push": W.config_push}[which](K=K, H=H)
    m = cfg.mppi
    ref = _mppi.Controller(cfg.robot, cfg.cost, m)
    ranks = [_mppi.Controller(cfg.robot, cfg.cost, m) for _ in range(world)]
    for c in [ref] + ranks:
        c.set_nominal(cfg.mu0)
    x0 = cfg.x0.astype(np.float32)
    for step in range(3):
        nominal = ref.get_nominal().copy()
        u0_ref, mu_ref = np.zeros(12, np.float32), np.zeros(48, np.float32)
        assert ref.step(x0, step, u0_out=u0_ref, mu_out=mu_ref) == 0
        parts, Us, Ls = [], [], []
        for r, c in enumerate(ranks):
            k0, n = SH.shard_range(K, r, world)
            parts.append(c.step_partial(x0, step, k0, n))
            U, L = c.last_samples()
            Us.append(U[:n])
            Ls.append(L[:n])
        Lmin = min(p[0] for p in parts)
        rmin = lambda v: Lmin  # noqa: E731  (the all-reduce(min) of every rank's m)
        total = sum(math.exp(-(p[0] - Lmin) / m["lam"]) * p[1:] for p in parts)
        rsum = lambda a: total  # noqa: E731  (the all-reduce(sum))
        mus = []
        for r, c in enumerate(ranks):
            k0, n = SH.shard_range(K, r, world)
            sums = SH.combine(parts[r], c.lam, rmin, rsum)
            u0, mu = np.zeros(12, np.float32), np.zeros(48, np.float32)
            assert c.step_finalize(sums, u0, mu) == 0
            assert np.array_equal(u0, mu[:12])
            mus.append(mu)
        for mu in mus[1:]:
            assert np.array_equal(mu, mus[0])
        U_all, L_all = np.concatenate(Us), np.concatenate(Ls)
        assert np.array_equal(U_all.view(np.uint32), O.sample(m, nominal, step).view(np.uint32))
        _, mu_o, _ = O.update(L_all, U_all, m["lam"])
        assert rel(mus[0], mu_o) <= 1e-6, step
        assert rel(mus[0], mu_ref) <= 1e-6, step
        sh = O.shift(mus[0], H, m["ctrl_steps"])
        for c in ranks:
            assert rel(c.get_nominal(), sh) <= 1e-6
    for c in [ref] + ranks:
        c.close()


def test_sharded_step_range_checks_and_no_finite_cost():
    cfg = W.config_stand(K=32, H=12)
    c = _mppi.Controller(cfg.robot, cfg.cost, cfg.mppi)
    c.set_nominal(cfg.mu0)
    x0 = cfg.x0.astype(np.float32)
    for k0, n in [(-1, 4), (0, 0), (30, 3)]:
        with pytest.raises(_mppi.MppiError):
            c.step_partial(x0, 0, k0, n)
    # every cost non-finite: the shard reports no minimum and zero sums; the
    # finalize keeps the mean and reports NONFINITE
    bad = _mppi.Controller(cfg.robot, dict(cfg.cost, w_z=float("inf")), cfg.mppi)
    bad.set_nominal(cfg.mu0)
    p = bad.step_partial(x0, 0, 0, 32)
    assert math.isinf(p[0]) and np.all(p[1:] == 0)
    mu = np.zeros(48, np.float32)
    assert bad.step_finalize(p[1:], mu_out=mu, check=False) == _mppi.MPPI_ERR_NONFINITE
    assert np.array_equal(mu, cfg.mu0.astype(np.float32))
    c.close()
    bad.close()
