"""Pins of the spline (Sec. III-B, Fig. 2), the softmax update (Eq. 1, Eq. 2),
the shift of Alg. 1 and the L_walk / L_box costs (Sec. IV-B, IV-D) of the
oracle, against closed forms and limits."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W


def cubic_knots(coef):
    """Knots (at tau = j/3) of per-joint cubics p(tau) = sum c_k tau^k."""
    taus = np.arange(4) / 3
    U = np.zeros((4, 12))
    for j in range(4):
        U[j] = sum(coef[k] * taus[j] ** k for k in range(4))
    return U.astype(np.float32), coef


def test_spline_reproduces_cubics():
    rng = np.random.default_rng(0)
    coef = rng.normal(size=(4, 12))
    U, _ = cubic_knots(coef)
    Ud = U.astype(np.float64)
    # refit the polynomial through the stored float knots exactly
    taus = np.arange(4) / 3
    V = np.vander(taus, 4, increasing=True)
    c = np.linalg.solve(V, Ud)
    for tau in np.linspace(0, 1, 37):
        ref = sum(c[k] * tau ** k for k in range(4))
        assert np.allclose(O.spline_eval(U.ravel(), tau), ref, atol=1e-12)


@pytest.mark.parametrize("H", [2, 5, 50, 100, 151])
def test_spline_basis_partition_and_knots(H):
    for t in range(H):
        B = O.spline_basis(H, t)
        assert B.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.allclose(O.spline_basis(H, 0), [1, 0, 0, 0], atol=1e-15)
    assert np.allclose(O.spline_basis(H, H - 1), [0, 0, 0, 1], atol=1e-15)
    if (H - 1) % 3 == 0:
        assert np.allclose(O.spline_basis(H, (H - 1) // 3), [0, 1, 0, 0], atol=1e-14)


def test_shift_of_polynomial_knots():
    """Shifting re-samples the cubic at tau_j + delta; past tau = 1 it holds p(1)."""
    rng = np.random.default_rng(1)
    coef = rng.normal(size=(4, 12)) * 0.3
    U, _ = cubic_knots(coef)
    taus = np.arange(4) / 3
    c = np.linalg.solve(np.vander(taus, 4, increasing=True), U.astype(np.float64))
    H, cs = 100, 2
    d = cs / (H - 1)
    out = O.shift(U.ravel(), H, cs).reshape(4, 12)
    for j in range(4):
        tau = min(taus[j] + d, 1.0)
        ref = sum(c[k] * tau ** k for k in range(4))
        assert np.allclose(out[j], ref, atol=2e-7)
    const = np.tile(W.stand_mu()[:12], 4)
    assert np.array_equal(O.shift(const, 50, 1), const)


def test_update_lambda_limits_and_invariants():
    rng = np.random.default_rng(2)
    K = 8
    U = rng.normal(size=(K, 48)).astype(np.float32)
    L = rng.uniform(0, 10, K).astype(np.float32)
    # lambda -> 0: the argmin sample (Fig. 2 reading)
    _, mu0, w0 = O.update(L, U, 1e-6)
    assert np.array_equal(mu0, U[np.argmin(L)])
    # lambda -> infinity: the sample mean
    _, muinf, winf = O.update(L, U, 1e12)
    assert np.allclose(muinf, U.astype(np.float64).mean(0), atol=1e-6)
    assert np.allclose(winf, 1 / K, atol=1e-12)
    # weights sum to one, are invariant to a cost offset
    _, mu1, w1 = O.update(L, U, 0.7)
    assert w1.sum() == pytest.approx(1.0, abs=1e-15)
    _, mu2, w2 = O.update(L.astype(np.float64) + 64.0, U, 0.7, double_costs=True)
    assert np.allclose(w1, w2, rtol=1e-12)
    # brute force: Eq. 1 and Eq. 2 with exp in long double (math.fsum sums)
    ex = [math.exp(-(float(l) - float(L.min())) / 0.7) for l in L]
    Z = math.fsum(ex)
    ref = np.array([math.fsum(ex[k] / Z * float(U[k, d]) for k in range(K)) for d in range(48)])
    assert np.allclose(mu1, ref, rtol=1e-6, atol=1e-7)


def test_update_nonfinite():
    U = np.ones((4, 48), np.float32) * np.arange(4, dtype=np.float32)[:, None]
    L = np.array([np.nan, 3.0, np.inf, 5.0], np.float32)
    rc, mu, w = O.update(L, U, 1e-6)
    assert rc == 0 and np.allclose(mu, 1.0) and w[0] == 0 and w[2] == 0
    rc, _, _ = O.update(np.array([np.nan] * 4, np.float32), U, 0.1)
    assert rc == -1


def test_mppi_step_degenerate_cases():
    cfg = W.config_stand(K=1, H=20)
    w = O.World(cfg.robot)
    mu = cfg.mu0 + np.float32(0.01)
    rc, mu1, u0, L, U = O.mppi_step(w, cfg.cost, cfg.mppi, cfg.x0, mu, 0)
    # K = 1: only the nominal sample, so mu' = mu, u0 = mu[0], then the shift
    assert rc == 0 and np.array_equal(u0, mu[:12])
    assert np.array_equal(mu1, O.shift(mu, 20, 1))
    # sigma = 0: every sample equals mu
    cfg = W.config_stand(K=16, H=20)
    cfg.mppi["sigma"][:] = 0
    rc, mu2, u0, L, U = O.mppi_step(w, cfg.cost, cfg.mppi, cfg.x0, mu, 0)
    assert np.array_equal(u0, mu[:12]) and np.allclose(L, L[0])


def test_cost_closed_forms():
    w = O.World(W.robot())
    c = W.cost("stand")
    x = W.stand_state(z=0.3)
    u = np.tile(W.STAND, 4)
    assert O.stage_cost(w, c, x, u, 0.0) == pytest.approx(0.0, abs=1e-15)
    x2 = x.copy()
    x2[2] = 0.25
    assert O.stage_cost(w, c, x2, u, 0.0) == pytest.approx(1e3 * 0.05 ** 2, rel=1e-12)
    a = 0.3
    x3 = x.copy()
    x3[3:7] = [math.cos(a / 2), math.sin(a / 2), 0, 0]
    assert O.stage_cost(w, c, x3, u, 0.0) == pytest.approx(1e2 * 4 * math.sin(a / 2) ** 2, rel=1e-12)
    x3[3:7] = -x3[3:7]  # same attitude, other quaternion sign
    assert O.stage_cost(w, c, x3, u, 0.0) == pytest.approx(1e2 * 4 * math.sin(a / 2) ** 2, rel=1e-12)
    u2 = u + 0.1
    assert O.stage_cost(w, c, x, u2, 0.0) == pytest.approx(12 * 0.01, rel=1e-12)
    ct = W.cost("trot")
    x4 = x.copy()
    x4[22] = 0.2
    uref = O.gait_ref(ct, 0.1)
    assert O.stage_cost(w, ct, x4, uref, 0.1) == pytest.approx(1e2 * 0.3 ** 2, rel=1e-12)


def test_trot_reference_gait():
    ct = W.cost("trot")
    for t in np.linspace(0, 1, 17):
        r = O.gait_ref(ct, t).reshape(4, 3)
        assert np.allclose(O.gait_ref(ct, t + 0.5), O.gait_ref(ct, t), atol=1e-12)  # period
        assert np.allclose(r[0], r[3]) and np.allclose(r[1], r[2])  # diagonal pairs
        r2 = O.gait_ref(ct, t + 0.25).reshape(4, 3)
        assert np.allclose(r[0], r2[1], atol=1e-12)  # pairs half a period apart
        assert np.all(r[:, 2] <= W.STAND[2] + 1e-15)  # knee only flexes further


def test_box_cost_l1():
    w = O.World(W.robot(box=True))
    c = W.cost("push", box_goal=(1.6, 0.3))
    c["w_p"] = 0.0
    x = W.stand_state(z=0.3, box_xy=(0.6, -0.2))
    u = np.tile(W.STAND, 4)
    uref = O.gait_ref(c, 0.0)
    L = O.stage_cost(w, c, x, uref, 0.0)
    assert L == pytest.approx(1e2 * (1.0 + 0.5), rel=1e-12)


def test_closed_loop_stand_stays_up():
    """Integration check (not a parity pin): plain MPPI keeps the trunk up."""
    cfg = W.config_stand(K=64, H=30)
    w = O.World(cfg.robot)
    m = cfg.mppi
    x, mu = cfg.x0.copy(), cfg.mu0.copy()
    for s in range(15):
        rc, mu, u0, L, U = O.mppi_step(w, cfg.cost, m, x, mu, s)
        for _ in range(m["n_sub"]):
            x = O.substep(w, x, u0.astype(np.float64), m["dt"] / m["n_sub"])
    assert rc == 0 and x[2] > 0.25
