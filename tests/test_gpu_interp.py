"""GPU parity (through the C ABI) of the control representations of the
sampling ablation (Sec. III-B, Fig. 5) against the FP64 oracle: zeroth-order
hold, linear and cubic knots, and direct per-step targets.

Bounds as for the cubic path: samples bit-exact; rollout cost <= 1e-3 relative
on flat ground; update and shift <= 1e-6 relative given the same FP32 costs and
samples."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import _mppi, workloads as W  # noqa: E402

MODES = ["zero", "linear", "cubic", "direct"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def ctl_for(cfg, **kw):
    m = dict(cfg.mppi)
    m.update(kw)
    return _mppi.Controller(cfg.robot, cfg.cost, m), m


def nominal(m, mu48, rng=None):
    """a nominal of the representation's dimension around the 48 knots"""
    Dm = O.param_dim(m)
    mu = np.tile(mu48[:12], Dm // 12).astype(np.float32)
    n = min(48, Dm)
    mu[:n] = mu48[:n]
    if rng is not None:
        mu += (0.03 * rng.standard_normal(Dm)).astype(np.float32)
    return mu


@pytest.mark.parametrize("mode", MODES)
def test_param_dim_and_sample_bit_exact(mode):
    cfg = W.config_trot(K=300, H=40)
    ctl, m = ctl_for(cfg, interp=mode)
    Dm = O.param_dim(m)
    assert ctl.D == Dm == (480 if mode == "direct" else 48)
    mu = nominal(m, W.stand_mu(), np.random.default_rng(1))
    ctl.set_nominal(mu)
    assert np.array_equal(ctl.get_nominal(), mu)
    U = torch.empty((300, Dm), device="cuda")
    ctl.sample(5, out=U)
    Uo = O.sample(m, mu, 5)
    assert np.array_equal(U.cpu().numpy().view(np.uint32), Uo.view(np.uint32))


@pytest.mark.parametrize("which", ["stand", "trot"])
@pytest.mark.parametrize("mode", MODES)
def test_rollout_cost_parity(mode, which):
    if which == "stand":
        cfg, K, H, t0 = W.config_stand(), 64, 40, 0.0
    else:
        cfg, K, H, t0 = W.config_trot(), 64, 61, 0.37
    ctl, m = ctl_for(cfg, K=K, H=H, interp=mode)
    ctl.set_nominal(nominal(m, cfg.mu0))
    U = torch.empty((K, ctl.D), device="cuda")
    ctl.sample(0, out=U)
    L = torch.empty(K, device="cuda")
    x0 = cfg.x0.astype(np.float32)
    ctl.rollouts(dev(x0), U=U, n=K, t0=t0, L_out=L)
    Lo = O.rollouts(O.World(cfg.robot), cfg.cost, m, t0, x0.astype(np.float64), U.cpu().numpy())
    Lg = L.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(Lg))
    rel = np.abs(Lg - Lo) / np.maximum(np.abs(Lo), 1.0)
    assert rel.max() <= 1e-3, (mode, rel.max())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("K,H,lam", [(7, 12, 1e6), (513, 40, 0.05), (4096, 100, 0.1), (1000, 50, 0.2)])
def test_update_and_shift_parity(mode, K, H, lam):
    cfg = W.config_trot()
    ctl, m = ctl_for(cfg, K=K, H=H, lam=lam, interp=mode)
    Dm = ctl.D
    rng = np.random.default_rng(K)
    U = (np.tile(nominal(m, W.stand_mu()), (K, 1)) + rng.normal(0, 0.3, (K, Dm))).astype(np.float32)
    L = (100 + 5 * rng.random(K)).astype(np.float32)
    mu_g = torch.empty(Dm, device="cuda")
    u0_g = torch.empty(12, device="cuda")
    assert ctl.update(dev(L), dev(U), n=K, mu_out=mu_g, u0_out=u0_g) == 0
    _, mu_o, _ = O.update(L, U, lam, dim=Dm)
    mg = mu_g.cpu().numpy()
    e = np.abs(mg - mu_o) / np.maximum(np.abs(mu_o), 1)
    assert e.max() <= 1e-6, (mode, e.max())
    assert np.array_equal(u0_g.cpu().numpy(), mg[:12])
    sh = O.shift(mg, H, m["ctrl_steps"], mode)
    assert np.abs(ctl.get_nominal() - sh).max() <= 1e-6 * max(1.0, np.abs(sh).max())


@pytest.mark.parametrize("mode", MODES)
def test_update_nonfinite_keeps_and_shifts_the_mean(mode):
    cfg = W.config_stand()
    ctl, m = ctl_for(cfg, K=8, H=20, interp=mode)
    mu = nominal(m, W.stand_mu(), np.random.default_rng(4))
    ctl.set_nominal(mu)
    U = np.tile(mu, (8, 1))
    mu_h = np.zeros(ctl.D, np.float32)            # a host output makes the call report the status
    rc = ctl.update(dev(np.full(8, np.nan, np.float32)), dev(U), n=8, mu_out=mu_h)
    assert rc == _mppi.MPPI_ERR_NONFINITE
    assert np.array_equal(mu_h, mu)
    assert np.abs(ctl.get_nominal() - O.shift(mu, 20, m["ctrl_steps"], mode)).max() <= 1e-6


@pytest.mark.parametrize("mode", MODES)
def test_full_step_matches_the_oracle_update(mode):
    """mppi_step = sample -> rollouts -> update for every representation; the
    update of the GPU's own costs matches the oracle's on the same samples."""
    cfg = W.config_stand(K=64, H=30)
    ctl, m = ctl_for(cfg, interp=mode)
    mu = nominal(m, cfg.mu0)
    ctl.set_nominal(mu)
    u0 = np.zeros(12, np.float32)
    mu_upd = np.zeros(ctl.D, np.float32)
    ctl.step(cfg.x0.astype(np.float32), 2, u0_out=u0, mu_out=mu_upd)
    U_o = O.sample(m, mu, 2)
    ctl2, _ = ctl_for(cfg, interp=mode)
    L = torch.empty(64, device="cuda")
    ctl2.rollouts(dev(cfg.x0), U=dev(U_o), n=64, t0=2 * m["ctrl_steps"] * m["dt"], L_out=L)
    _, mu_same, _ = O.update(L.cpu().numpy(), U_o, m["lam"], dim=ctl.D)
    assert np.abs(mu_upd - mu_same).max() <= 1e-6 * max(1.0, np.abs(mu_same).max())
    assert np.array_equal(u0, mu_upd[:12])


def test_invalid_configurations():
    cfg = W.config_stand(K=16, H=20)
    with pytest.raises(_mppi.MppiError):
        ctl_for(cfg, interp=4)
    with pytest.raises(_mppi.MppiError):
        ctl_for(cfg, interp="direct", n_prop=4)      # the proposal is a 48-knot mean


def test_batch_runs_knot_representations_and_rejects_direct():
    cfg = W.config_stand(K=96, H=30)
    x0s = np.zeros((3, 50), np.float32)
    x0s[:, :37] = cfg.x0
    singles, members = [], []
    for i, mode in enumerate(["zero", "linear", "cubic"]):
        a, _ = ctl_for(cfg, interp=mode, inst=i)
        b, _ = ctl_for(cfg, interp=mode, inst=i)
        singles.append(a)
        members.append(b)
    batch = _mppi.Batch(members)
    for step in range(3):
        u0b = torch.zeros((3, 12), device="cuda")
        batch.step(dev(x0s), np.full(3, step, np.uint32), u0s=u0b)
        for i, c in enumerate(singles):
            u0 = np.zeros(12, np.float32)
            c.step(x0s[i, :37], step, u0_out=u0)
            assert np.abs(u0b.cpu().numpy()[i] - u0).max() <= 1e-6 * max(1.0, np.abs(u0).max()), (i, step)
            nb, ns = members[i].get_nominal(), c.get_nominal()
            assert np.abs(nb - ns).max() <= 1e-6 * max(1.0, np.abs(ns).max()), (i, step)
    d, _ = ctl_for(cfg, interp="direct")
    with pytest.raises(_mppi.MppiError):
        _mppi.Batch([d])


@pytest.mark.parametrize("mode", ["cubic", "direct"])
def test_update_with_whole_chunks_non_finite(mode):
    """The update kernels take each chunk's cost minimum and rescale the chunks
    by exp(-(m_c - L_min)/lambda): chunks whose costs are all non-finite (m_c
    infinite) must drop out, the chunk holding L_min must weigh 1.  For the knots
    K = 1000 is 8 chunks of 125; chunks 1 and 4 are all inf / NaN, chunk 6 holds
    the minimum.  Direct targets chunk by 16 samples here, so the same ranges
    cover several whole chunks each."""
    cfg = W.config_trot()
    K, H, lam = 1000, 50, 0.1
    ctl, m = ctl_for(cfg, K=K, H=H, lam=lam, interp=mode)
    Dm = ctl.D
    rng = np.random.default_rng(11)
    U = (np.tile(nominal(m, W.stand_mu()), (K, 1)) + rng.normal(0, 0.3, (K, Dm))).astype(np.float32)
    L = (100 + 3 * rng.random(K)).astype(np.float32)
    L[125:250] = np.inf
    L[500:625] = np.nan
    L[777] = 98.0
    mu_g = torch.empty(Dm, device="cuda")
    u0_g = torch.empty(12, device="cuda")
    assert ctl.update(dev(L), dev(U), n=K, mu_out=mu_g, u0_out=u0_g) == 0
    _, mu_o, _ = O.update(L, U, lam, dim=Dm)
    mg = mu_g.cpu().numpy()
    e = np.abs(mg - mu_o) / np.maximum(np.abs(mu_o), 1)
    assert e.max() <= 1e-6, (mode, e.max())
    assert np.array_equal(u0_g.cpu().numpy(), mg[:12])


@pytest.mark.parametrize("K,H", [(1, 3), (64, 2), (64, 3), (300, 4), (5, 7), (2000, 300), (16384, 100)])
def test_direct_update_sizes(K, H):
    """Direct targets at the horizons where 12 H is below, at and far above the
    48 knot parameters (H = 300: two column tiles of 450 groups of 4), with
    fewer samples than a chunk's 16 and at the paper-scale K = 16384 (hundreds
    of chunks): update, u0 and shift against the oracle <= 1e-6"""
    cfg = W.config_trot()
    lam = 0.1
    ctl, m = ctl_for(cfg, K=K, H=H, lam=lam, interp="direct")
    Dm = ctl.D
    assert Dm == 12 * H
    rng = np.random.default_rng(H)
    mu = nominal(m, W.stand_mu(), rng)
    ctl.set_nominal(mu)
    U = (mu[None, :] + rng.normal(0, 0.3, (K, Dm))).astype(np.float32)
    L = (100 + 8 * rng.random(K)).astype(np.float32)
    mu_g = torch.empty(Dm, device="cuda")
    u0_g = torch.empty(12, device="cuda")
    assert ctl.update(dev(L), dev(U), n=K, mu_out=mu_g, u0_out=u0_g) == 0
    _, mu_o, _ = O.update(L, U, lam, dim=Dm)
    mg = mu_g.cpu().numpy()
    e = np.abs(mg - mu_o) / np.maximum(np.abs(mu_o), 1)
    assert e.max() <= 1e-6, e.max()
    assert np.array_equal(u0_g.cpu().numpy(), mg[:12])
    sh = O.shift(mg, H, m["ctrl_steps"], "direct")
    assert np.array_equal(ctl.get_nominal(), sh.astype(np.float32))
    # a second update on the same handle (the combine's counter re-armed)
    L2 = L[::-1].copy()
    assert ctl.update(dev(L2), dev(U), n=K, mu_out=mu_g) == 0
    _, mu_o2, _ = O.update(L2, U, lam, dim=Dm)
    assert (np.abs(mu_g.cpu().numpy() - mu_o2) / np.maximum(np.abs(mu_o2), 1)).max() <= 1e-6


def test_direct_update_more_samples_than_k():
    """Device costs and targets of more samples than the handle's K: the row kernel's
    chunk count is capped independently of n, so the update takes any n"""
    cfg = W.config_trot()
    ctl, m = ctl_for(cfg, K=64, H=7, lam=0.2, interp="direct")
    n = 5000
    rng = np.random.default_rng(77)
    mu = nominal(m, W.stand_mu(), rng)
    ctl.set_nominal(mu)
    U = (mu[None, :] + rng.normal(0, 0.3, (n, ctl.D))).astype(np.float32)
    L = (50 + 4 * rng.random(n)).astype(np.float32)
    mu_g = torch.empty(ctl.D, device="cuda")
    assert ctl.update(dev(L), dev(U), n=n, mu_out=mu_g) == 0
    _, mu_o, _ = O.update(L, U, 0.2, dim=ctl.D)
    assert (np.abs(mu_g.cpu().numpy() - mu_o) / np.maximum(np.abs(mu_o), 1)).max() <= 1e-6
