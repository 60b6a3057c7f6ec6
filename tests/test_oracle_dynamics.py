"""Pins of the oracle's rigid-body dynamics against closed forms and
independent algorithms (CRBA + RNEA), invariants and limits.

The simulator replaces the paper's MuJoCo rollouts (arXiv 2409.10469,
Sec. III-A); these pins fix the project's own model, not MuJoCo's.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W


def quad_tree(g=9.81):
    r = W.robot()
    r["gravity"] = g
    w = O.World(r)
    return w, O.world_tree(w)


@pytest.mark.parametrize("seed", range(6))
def test_aba_matches_crba_solve(seed):
    """ABA equals the solve (M + diag(a)) qdd = tau - C (CRBA for M, RNEA for C)."""
    w, T = quad_tree()
    rng = np.random.default_rng(seed)
    x = W.random_states(1, seed, spread=3.0)[0]
    q, v = x[:19], x[19:]
    tau = rng.normal(0, 5, 12)
    arm = rng.uniform(0, 0.02, 12)
    fext = np.zeros((16, 6))
    fext[:13] = rng.normal(0, 3, (13, 6))
    acc = T.aba(q, v, tau, fext, arm)
    M = T.crba(q, arm)
    Cb = T.rnea(q, v, np.zeros(18), fext, arm)
    ref = np.linalg.solve(M, np.r_[np.zeros(6), tau] - Cb)
    assert np.max(np.abs(acc - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("seed", range(4))
def test_rnea_inverts_aba(seed):
    """RNEA(q, v, ABA(tau)) returns tau on the joints and zero base wrench."""
    w, T = quad_tree()
    rng = np.random.default_rng(100 + seed)
    x = W.random_states(1, 100 + seed, spread=2.0)[0]
    tau = rng.normal(0, 5, 12)
    arm = rng.uniform(0, 0.02, 12)
    acc = T.aba(x[:19], x[19:], tau, None, arm)
    out = T.rnea(x[:19], x[19:], acc, None, arm)
    assert np.max(np.abs(out[:6])) < 1e-10
    assert np.max(np.abs(out[6:] - tau)) < 1e-10


def test_mass_matrix_spd():
    w, T = quad_tree()
    for x in W.random_states(5, 7, spread=3.0):
        M = T.crba(x[:19])
        assert np.allclose(M, M.T, atol=1e-14)
        assert np.linalg.eigvalsh(M).min() > 0
        # total mass appears in the base linear block
        assert np.allclose(np.diag(M)[3:6], 12.0, atol=1e-12)


def test_momentum_rate_is_gravity():
    """sum of I a + v x* I v over bodies = external forces: with gravity only, the
    world momentum rate is the weight, applied at the centre of mass."""
    for g in (0.0, 9.81):
        w, T = quad_tree(g)
        for x in W.random_states(4, 11, spread=3.0):
            q, v = x[:19], x[19:]
            tau = np.random.default_rng(1).normal(0, 5, 12)
            acc = T.aba(q, v, tau)
            hd = T.momentum_rate(q, v, acc)
            R, p = T.fk(q)
            masses = [5.2] + [0.5, 1.0, 0.2] * 4
            # centre of mass of every body in world: body origin + R com
            coms = []
            for i in range(13):
                com_b = np.zeros(3)
                if i > 0 and (i - 1) % 3 == 1:
                    com_b = np.array([0, 0, -0.1065])
                if i > 0 and (i - 1) % 3 == 2:
                    com_b = np.array([0, 0, -0.1065])
                coms.append(p[i] + R[i] @ com_b)
            M = sum(masses)
            c = sum(m * cc for m, cc in zip(masses, coms)) / M
            F = np.array([0, 0, -M * g])
            assert np.allclose(hd[3:], F, atol=1e-10)
            assert np.allclose(hd[:3], np.cross(c, F), atol=1e-10)


def test_zero_gravity_flight_momentum_drift_first_order():
    """Contact-free flight in zero gravity under internal PD torques: momentum is
    conserved by the dynamics; the semi-implicit discretisation drifts O(h)."""
    r = W.robot()
    r["gravity"] = 0.0
    w = O.World(r)
    T = O.world_tree(w)
    x0 = W.stand_state(z=5.0)
    x0[7:19] += np.random.default_rng(3).uniform(-0.4, 0.4, 12)
    x0[19:25] = [0.5, -0.3, 0.2, 0.1, 0.0, 0.3]
    u = np.tile(W.STAND, 4)
    drifts = []
    for h in (2e-3, 1e-3, 5e-4):
        x = x0.copy()
        h0 = T.momentum(x[:19], x[19:])
        for _ in range(int(round(0.2 / h))):
            x = O.substep(w, x, u, h)
        h1 = T.momentum(x[:19], x[19:])
        drifts.append(np.max(np.abs(h1 - h0)))
    # linear momentum is exactly conserved by v += h a (sum of internal forces 0)
    assert drifts[0] < 1e-2
    assert 1.6 < drifts[0] / drifts[1] < 2.5 and 1.6 < drifts[1] / drifts[2] < 2.5


def pendulum(m, L, fixed_axis=1):
    """Rod of mass m, length L hanging from a revolute joint at the origin."""
    T = O.Tree(floating=False, gz=-9.81)
    Ic = np.diag([m * L * L / 12, m * L * L / 12, 0.0])
    T.add(-1, fixed_axis, [0, 0, 0], m, [0, 0, -L / 2], Ic)
    return T


def test_single_pendulum_acceleration_closed_form():
    m, L = 1.3, 0.7
    T = pendulum(m, L)
    Ipiv = m * L * L / 3
    for th in np.linspace(-3, 3, 13):
        acc = T.aba([th], [0.4], [0.0])
        assert acc[0] == pytest.approx(-m * 9.81 * (L / 2) * math.sin(th) / Ipiv, abs=1e-12)


def test_double_pendulum_closed_form():
    """Two point-like masses (tiny rods) on massless links: textbook equations
    M(q) qdd + C(q, qd) + G(q) = tau of the planar double pendulum."""
    m1, m2, l1, l2, g = 1.0, 0.7, 0.5, 0.4, 9.81
    T = O.Tree(floating=False, gz=-g)
    eps = 1e-9
    T.add(-1, 1, [0, 0, 0], m1, [0, 0, -l1], np.eye(3) * eps)
    T.add(0, 1, [0, 0, -l1], m2, [0, 0, -l2], np.eye(3) * eps)
    rng = np.random.default_rng(5)
    for _ in range(10):
        q = rng.uniform(-2, 2, 2)
        qd = rng.uniform(-3, 3, 2)
        tau = rng.uniform(-2, 2, 2)
        acc = T.aba(q, qd, tau)
        # rotation about +y: a mass at -l z rotated by q has position (-l sin q, -l cos q) in (x, z)
        c2 = math.cos(q[1])
        s2 = math.sin(q[1])
        M = np.array([[m1 * l1 ** 2 + m2 * (l1 ** 2 + l2 ** 2 + 2 * l1 * l2 * c2),
                       m2 * (l2 ** 2 + l1 * l2 * c2)],
                      [m2 * (l2 ** 2 + l1 * l2 * c2), m2 * l2 ** 2]])
        h = m2 * l1 * l2 * s2
        Cv = np.array([-h * (2 * qd[0] * qd[1] + qd[1] ** 2), h * qd[0] ** 2])
        G = np.array([(m1 + m2) * g * l1 * math.sin(q[0]) + m2 * g * l2 * math.sin(q[0] + q[1]),
                      m2 * g * l2 * math.sin(q[0] + q[1])])
        ref = np.linalg.solve(M, tau - Cv - G)
        assert np.allclose(acc, ref, rtol=1e-6, atol=1e-6)


def _period(T, th0, h):
    """Period from successive upward zero crossings of the angle, semi-implicit Euler."""
    q, qd, t = th0, 0.0, 0.0
    crossings = []
    prev = q
    while len(crossings) < 3 and t < 20:
        a = T.aba([q], [qd], [0.0])[0]
        qd += h * a
        q += h * qd
        t += h
        if prev < 0 <= q:
            crossings.append(t - h * q / (q - prev))
        prev = q
    return crossings[2] - crossings[1]


def test_pendulum_period_small_and_large_amplitude():
    m, L, g = 1.0, 0.5, 9.81
    T = pendulum(m, L)
    Ipiv, d = m * L * L / 3, L / 2
    w0 = math.sqrt(m * g * d / Ipiv)
    # small amplitude: 2 pi / w0
    assert _period(T, 0.01, 1e-4) == pytest.approx(2 * math.pi / w0, rel=2e-4)
    # large amplitude: 4 K(k) / w0, k = sin(th0 / 2), K by the AGM
    th0 = 2.0
    k = math.sin(th0 / 2)
    a, b = 1.0, math.sqrt(1 - k * k)
    for _ in range(30):
        a, b = (a + b) / 2, math.sqrt(a * b)
    Kk = math.pi / (2 * a)
    ref = 4 * Kk / w0
    errs = [abs(_period(T, th0, h) - ref) for h in (4e-4, 2e-4, 1e-4)]
    assert errs[-1] < 2e-4 * ref
    assert errs[0] > errs[1] > errs[2]


def test_free_fall_exact():
    """No contact, no PD, joints at rest: every body falls together and the trunk
    height follows z_n = z0 - g h^2 n (n + 1) / 2 exactly (semi-implicit Euler)."""
    r = W.robot()
    r["kp"], r["kd"] = 0.0, 0.0
    r["armature"] = 0.01
    w = O.World(r)
    x = W.stand_state(z=10.0)
    u = np.tile(W.STAND, 4)
    h = 1e-3
    for n in range(1, 201):
        x = O.substep(w, x, u, h)
        assert x[2] == pytest.approx(10.0 - 9.81 * h * h * n * (n + 1) / 2, abs=1e-11)
    assert np.allclose(x[7:19], np.tile(W.STAND, 4), atol=1e-11)
    assert np.allclose(x[3:7], [1, 0, 0, 0], atol=1e-12)


def box_world(**kw):
    r = W.robot(box=True, **kw)
    return O.World(r), r


def robot_far(x):
    x[0] = 50.0
    return x


def test_box_rest_penetration_mg_over_k():
    """Free box at rest on a plane: its 4 bottom corner spheres carry mg/4 each,
    penetration mg / (4 k), and the contact force balances the weight."""
    w, r = box_world()
    m, k = r["box_mass"], r["k_contact"]
    pen = m * 9.81 / (4 * k)
    x = robot_far(W.stand_state(box_xy=(0.0, 0.0)))
    x[39] = r["box_size"][2] / 2 + r["box_corner_r"] - pen
    _, fbox = O.contact_fext(w, x)
    assert fbox[3:] == pytest.approx([0, 0, m * 9.81], abs=1e-9)
    assert np.allclose(fbox[:3], 0, atol=1e-9)
    # and the simulated box settles there
    x[39] += 0.002
    u = np.tile(W.STAND, 4)
    for _ in range(3000):
        x = O.substep(w, x, u, 1e-3)
    assert x[39] == pytest.approx(r["box_size"][2] / 2 + r["box_corner_r"] - pen, abs=1e-7)


def test_box_sliding_friction_deceleration():
    """Sliding at |v| >> eps_v: friction decelerates at mu g |v| / sqrt(|v|^2 + eps^2)."""
    w, r = box_world()
    m, k, mu, eps = r["box_mass"], r["k_contact"], r["mu"], r["eps_v"]
    pen = m * 9.81 / (4 * k)
    x = robot_far(W.stand_state(box_xy=(0.0, 0.0)))
    x[39] = r["box_size"][2] / 2 + r["box_corner_r"] - pen
    vx = 1.5
    x[37 + 13 - 6 + 3] = vx  # box body-frame linear velocity x
    _, fbox = O.contact_fext(w, x)
    assert fbox[3] == pytest.approx(-mu * m * 9.81 * vx / math.sqrt(vx * vx + eps * eps), rel=1e-12)
    assert fbox[5] == pytest.approx(m * 9.81, rel=1e-12)


def test_heightfield_reproduces_a_plane():
    """A heightfield sampled from a plane interpolates it exactly, with the plane's
    gradient and the contact normal (-a, -b, 1)/|.|."""
    a, b, c = 0.13, -0.07, 0.02
    n = 16
    xs = np.arange(n) * 0.05
    X, Y = np.meshgrid(xs, xs)
    hf = (a * X + b * Y + c).astype(np.float64)
    r = W.robot("heightfield", heightfield=hf.astype(np.float32), hf_cell=0.05)
    # float32 storage: compare against the stored values' plane within float rounding
    w = O.World(r)
    rng = np.random.default_rng(0)
    for _ in range(50):
        px, py = rng.uniform(0.01, 0.74, 2)
        h, hx, hy = O.terrain_height(w, px, py)
        assert h == pytest.approx(a * px + b * py + c, abs=1e-7)
        assert hx == pytest.approx(a, abs=1e-5) and hy == pytest.approx(b, abs=1e-5)
    # outside the grid: clamped height, zero slope across the clamped edge
    h, hx, hy = O.terrain_height(w, -1.0, 0.3)
    assert hx == 0.0 and h == pytest.approx(b * 0.3 + c, abs=1e-7)


def test_static_box_contact_normal_and_depth():
    r = W.robot(static_boxes=[((1.0, -0.5, 0.0), (1.5, 0.5, 0.3))])
    w = O.World(r)
    x = robot_far(W.stand_state(z=5.0))
    # put the trunk (centre sphere at the trunk origin) just inside the box's top face
    x[0], x[1], x[2] = 1.2, 0.0, 0.3 + 0.055 - 0.004
    fext, _ = O.contact_fext(w, x)
    # the three trunk spheres (x = 0, +-0.15) touch the top face: force along +z,
    # k * pen each with zero velocity; pen from the model's (FP32-valued) top and radius
    pen = r["sbox_hi"][0][2] + r["trunk_sphere_r"] - x[2]
    assert abs(pen - 0.004) < 1e-7
    assert fext[0][5] == pytest.approx(3 * 2e4 * pen, rel=1e-9)
    # sphere centre inside the box leaves through the nearest face (x-hi here)
    x[0], x[2] = 1.49 + 0.15, 0.15
    fext, _ = O.contact_fext(w, x)
    assert fext[0][3] > 0


def test_implicit_pd_definition():
    """A sub-step realises the implicit PD law: the joint torque that RNEA needs for
    the step's acceleration equals kp (u - q_new) - kd qd_new at the END of the
    step (q_new = q + h qd_new), zero gravity and no contact."""
    r = W.robot()
    r["gravity"] = 0.0
    w = O.World(r)
    T = O.world_tree(w)
    x = W.random_states(1, 21, spread=2.0)[0]
    x[2] = 5.0
    u = np.tile(W.STAND, 4) + np.random.default_rng(2).uniform(-0.3, 0.3, 12)
    h = 1e-3
    xn = O.substep(w, x, u, h)
    acc = (xn[19:] - x[19:]) / h
    tau = T.rnea(x[:19], x[19:], acc)
    qd_new = xn[25:37]
    q_new = x[7:19] + h * qd_new
    expect = 30.0 * (u - q_new) - 1.0 * qd_new
    assert np.allclose(tau[6:], expect, atol=1e-7)
    assert np.allclose(tau[:6], 0, atol=1e-7)


def test_box_spinning_friction_torque():
    """Box at rest height spinning about z: every bottom corner slides at w r, so
    friction gives a yaw torque -4 mu (m g / 4) r |v| / sqrt(|v|^2 + eps^2)."""
    w, r = box_world()
    m, k, mu, eps = r["box_mass"], r["k_contact"], r["mu"], r["eps_v"]
    pen = m * 9.81 / (4 * k)
    x = robot_far(W.stand_state(box_xy=(0.0, 0.0)))
    x[39] = r["box_size"][2] / 2 + r["box_corner_r"] - pen
    wz = 2.0
    x[46] = wz
    _, fbox = O.contact_fext(w, x)
    rc = math.hypot(0.25, 0.25)
    v = wz * rc
    assert fbox[2] == pytest.approx(-mu * m * 9.81 * rc * v / math.sqrt(v * v + eps * eps), rel=1e-12)
    assert np.allclose(fbox[[0, 1, 3, 4]], 0, atol=1e-9)


def _cost_sensitivity(eps_v, n_sub, K=48):
    cfg = W.config_trot()
    cfg.robot["eps_v"] = eps_v
    m = dict(cfg.mppi, K=K, H=100, n_sub=n_sub)
    U = O.sample(m, cfg.mu0, 0)
    x0 = cfg.x0.astype(np.float32).astype(np.float64)
    w = O.World(cfg.robot)
    L = O.rollouts(w, cfg.cost, m, 0.0, x0, U)
    xp = x0 * (1 + 1e-7 * np.random.default_rng(0).standard_normal(x0.shape))
    Lp = O.rollouts(w, cfg.cost, m, 0.0, xp, U)
    return np.abs(Lp - L) / np.maximum(np.abs(L), 1)


def test_model_spec_rollouts_well_conditioned():
    """The spec's sub-step (h = 0.625 ms) and friction regularisation
    (eps_v = 0.3 m/s) keep the explicit contact terms inside the semi-implicit
    Euler stability limit: a 1e-7 relative change of x0 moves the H = 100 trot
    rollout costs by < 1e-4 (median < 1e-6).  With eps_v = 0.01 m/s and
    h = 1.25 ms the friction slope mu f_n / eps_v is ~30x past the limit, feet
    chatter in stick, and the same perturbation moves costs by percents."""
    r = W.robot()
    assert r["eps_v"] == 0.3 and W.n_sub_for(0.005) == 8 and W.n_sub_for(0.01) == 16
    good = _cost_sensitivity(0.3, 8)
    assert np.median(good) < 1e-6 and good.max() < 1e-4
    bad = _cost_sensitivity(0.01, 4)
    assert np.median(bad) > 1e-3
