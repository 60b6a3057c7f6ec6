"""Pins of the oracle's control representations (Sec. III-B; the sampling-
representation ablation of Fig. 5): zeroth-order hold, linear and cubic
interpolation of 4 knots at tau_j = j / 3, and direct sampling of one target per
dt step.  Each is checked against what its definition fixes."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W


@pytest.mark.parametrize("H", [2, 4, 7, 50, 100, 150])
def test_zeroth_order_basis(H):
    prev = 0
    for t in range(H):
        B = O.interp_basis("zero", H, t)
        j = int(np.argmax(B))
        assert np.array_equal(B, np.eye(4)[j])               # one knot held
        assert j == min(3, (3 * t) // (H - 1)) and j >= prev  # the knot at or before tau_t
        prev = j
    assert np.argmax(O.interp_basis("zero", H, H - 1)) == 3


@pytest.mark.parametrize("H", [2, 4, 7, 50, 100, 150])
def test_linear_basis_reproduces_lines(H):
    a, b = 0.3, -1.7
    knots = np.array([a + b * j / 3 for j in range(4)])
    for t in range(H):
        B = O.interp_basis("linear", H, t)
        assert B.min() >= 0 and abs(B.sum() - 1) < 1e-15
        assert np.count_nonzero(B) <= 2
        assert abs(B @ knots - (a + b * t / (H - 1))) < 1e-12
    # a knot time that falls on a dt step gives the knot itself
    if (H - 1) % 3 == 0:
        for j in range(4):
            assert np.array_equal(O.interp_basis("linear", H, j * (H - 1) // 3), np.eye(4)[j])


def test_controls_per_representation():
    rng = np.random.default_rng(1)
    H = 40
    U = rng.standard_normal(48).astype(np.float32)
    Ud = rng.standard_normal(12 * H).astype(np.float32)
    for t in (0, 7, 13, 39):
        for mode in ("zero", "linear", "cubic"):
            B = O.interp_basis(mode, H, t)
            np.testing.assert_allclose(O.controls(mode, H, t, U), B @ U.reshape(4, 12).astype(np.float64),
                                       rtol=0, atol=1e-12)
        assert np.array_equal(O.controls("direct", H, t, Ud), Ud[12 * t:12 * t + 12].astype(np.float64))
    # the cubic basis is the Lagrange basis the spline tests pin
    B = np.zeros(4)
    assert np.allclose(O.interp_basis("cubic", H, 5), O.interp_basis(0, H, 5))


def test_direct_sampling_shares_the_knot_noise():
    """Direct samples draw D = 12 H normals from the same Philox counters, so the
    first 48 coincide with the knot representation's (uniform sigma, same centre)."""
    cfg = W.config_trot(K=16, H=30)
    m = dict(cfg.mppi)
    m["sigma"] = [0.3] * 48
    mu = cfg.mu0.astype(np.float32)
    mud = np.tile(mu[:12], 30).astype(np.float32)
    mud[:48] = mu
    Uk = O.sample(m, mu, 3)
    Ud = O.sample(dict(m, interp="direct"), mud, 3)
    assert Ud.shape == (16, 360)
    assert np.array_equal(Ud[:, :48].view(np.uint32), Uk.view(np.uint32))
    assert np.array_equal(Ud[0], mud)                        # sample 0 is the nominal
    assert np.all(Ud[:, 0::3] >= m["q_lo"][0]) and np.all(Ud[:, 2::3] <= m["q_hi"][2])


def test_update_any_dimension_brute_force():
    rng = np.random.default_rng(2)
    for K, Dm in ((5, 48), (7, 120), (3, 1800)):
        L = rng.uniform(0, 3, K)
        U = rng.standard_normal((K, Dm)).astype(np.float32)
        lam = 0.7
        rc, mu, w = O.update(L, U, lam, dim=Dm)
        assert rc == 0
        wl = np.exp(-(np.longdouble(L) - np.longdouble(L.min())) / np.longdouble(lam))
        wl /= wl.sum()
        ref = (wl[:, None] * U.astype(np.longdouble)).sum(0)
        np.testing.assert_allclose(mu, ref.astype(np.float64), rtol=0, atol=2e-7)
        assert abs(w.sum() - 1) < 1e-15


def test_shift_direct():
    H, c = 10, 3
    mu = np.arange(12 * H, dtype=np.float32)
    out = O.shift(mu, H, c, "direct").reshape(H, 12)
    for t in range(H):
        assert np.array_equal(out[t], mu.reshape(H, 12)[min(t + c, H - 1)])


def test_shift_linear_of_a_line_and_zeroth_hold():
    a, b = 0.2, 0.9
    knots = np.repeat(np.array([a + b * j / 3 for j in range(4)], np.float32)[:, None], 12, 1).ravel()
    for H, c in ((100, 2), (100, 33), (4, 1), (50, 20)):
        out = O.shift(knots, H, c, "linear").reshape(4, 12)
        for j in range(4):
            tau = min(1.0, j / 3 + c / (H - 1))
            assert np.allclose(out[j], a + b * tau, atol=1e-6)
        z = O.shift(knots, H, c, "zero").reshape(4, 12)
        for j in range(4):
            src = min(3, j + (3 * c) // (H - 1))
            assert np.array_equal(z[j], knots.reshape(4, 12)[src])


@pytest.mark.parametrize("mode", ["zero", "linear", "cubic", "direct"])
def test_mppi_step_degenerate_cases_per_representation(mode):
    """K = 1: only the nominal is sampled, so mu' = shifted(mu); sigma = 0 the same."""
    cfg = W.config_stand(K=1, H=12)
    world = O.World(cfg.robot)
    m = dict(cfg.mppi, interp=mode)
    Dm = O.param_dim(m)
    rng = np.random.default_rng(3)
    mu = (np.tile(cfg.mu0[:12], Dm // 12) + 0.05 * rng.standard_normal(Dm)).astype(np.float32)
    for mm in (m, dict(m, K=6, sigma=[0.0] * 48)):
        rc, mu_new, u0, L, U = O.mppi_step(world, cfg.cost, mm, cfg.x0, mu, 0)
        assert rc == 0
        assert np.array_equal(u0, mu[:12])
        assert np.allclose(mu_new, O.shift(mu, mm["H"], mm["ctrl_steps"], mode), atol=1e-7)
