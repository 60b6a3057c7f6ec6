"""ctypes wrapper of the FP64 CPU oracle (liboracle.so).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs import this package.  The product path (the CUDA library and
its binding) never imports, loads or calls it, and the oracle imports nothing
from the product path: both are fed plain dicts and arrays.

Every function cites the passage of arXiv 2409.10469 it follows in the C
sources (oracle/*.c).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

NJ, D = 12, 48


class OrParams(C.Structure):
    _fields_ = [
        ("trunk_mass", C.c_double), ("trunk_size", C.c_double * 3),
        ("hip_x", C.c_double), ("hip_y", C.c_double), ("hip_z", C.c_double),
        ("abd_mass", C.c_double), ("abd_radius", C.c_double),
        ("thigh_offset_y", C.c_double),
        ("thigh_mass", C.c_double), ("thigh_length", C.c_double),
        ("calf_mass", C.c_double), ("calf_length", C.c_double),
        ("rod_radius", C.c_double), ("foot_radius", C.c_double),
        ("n_trunk_spheres", C.c_int), ("trunk_sphere_x", C.c_double * 4),
        ("trunk_sphere_r", C.c_double),
        ("gravity", C.c_double),
        ("kp", C.c_double), ("kd", C.c_double), ("armature", C.c_double),
        ("k_contact", C.c_double), ("c_contact", C.c_double), ("mu", C.c_double),
        ("eps_v", C.c_double),
        ("has_box", C.c_int), ("box_mass", C.c_double), ("box_size", C.c_double * 3),
        ("box_corner_r", C.c_double),
        ("terrain", C.c_int), ("hf_nx", C.c_int), ("hf_ny", C.c_int),
        ("hf_cell", C.c_double), ("hf_x0", C.c_double), ("hf_y0", C.c_double),
        ("hf", C.POINTER(C.c_float)),
        ("n_static_boxes", C.c_int), ("sbox_lo", (C.c_double * 3) * 4),
        ("sbox_hi", (C.c_double * 3) * 4),
    ]


class OrCost(C.Structure):
    _fields_ = [
        ("w_z", C.c_double), ("z_ref", C.c_double), ("w_o", C.c_double),
        ("w_v", C.c_double), ("v_ref", C.c_double),
        ("w_p", C.c_double), ("goal_xy", C.c_double * 2),
        ("w_u", C.c_double), ("w_box", C.c_double), ("box_goal_xy", C.c_double * 2),
        ("gait", C.c_int), ("gait_period", C.c_double), ("gait_hip_amp", C.c_double),
        ("gait_knee_amp", C.c_double), ("stand", C.c_double * 3), ("w_terminal", C.c_double),
        ("raibert_k", C.c_double), ("raibert_len", C.c_double), ("z_rel", C.c_int),
    ]


class OrMppi(C.Structure):
    _fields_ = [
        ("K", C.c_int), ("H", C.c_int), ("n_sub", C.c_int), ("ctrl_steps", C.c_int),
        ("dt", C.c_double), ("lam", C.c_double),
        ("sigma", C.c_float * 48), ("q_lo", C.c_float * 3), ("q_hi", C.c_float * 3),
        ("seed", C.c_uint64), ("inst", C.c_uint32), ("n_prop", C.c_int), ("interp", C.c_int),
    ]


# control representations (oracle.h OR_INTERP_*)
INTERP = {"cubic": 0, "zero": 1, "linear": 2, "direct": 3}


def param_dim(m: dict) -> int:
    """Parameters per sample: 48 knots, or 12 targets per dt step (direct)."""
    return NJ * m["H"] if interp_of(m) == 3 else D


def interp_of(m: dict) -> int:
    v = m.get("interp", 0)
    return INTERP[v] if isinstance(v, str) else int(v)


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, fp = C.POINTER(C.c_double), C.POINTER(C.c_float)
        u32p = C.POINTER(C.c_uint32)
        L.or_world_size.restype = C.c_size_t
        L.or_tree_size.restype = C.c_size_t
        L.or_world_init.argtypes = [C.c_void_p, C.POINTER(OrParams)]
        L.or_rollout.restype = C.c_double
        L.or_rollout.argtypes = [C.c_void_p, C.POINTER(OrCost), C.c_int, C.c_int, C.c_double,
                                 C.c_double, dp, fp, dp]
        L.or_rollouts.argtypes = [C.c_void_p, C.POINTER(OrCost), C.POINTER(OrMppi), C.c_double,
                                  dp, C.c_int, fp, C.c_int, dp, dp, C.c_int]
        L.or_substep.argtypes = [C.c_void_p, dp, dp, C.c_double]
        L.or_contact_fext.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_stage_cost.restype = C.c_double
        L.or_stage_cost.argtypes = [C.c_void_p, C.POINTER(OrCost), dp, dp, C.c_double]
        L.or_terminal_cost.restype = C.c_double
        L.or_terminal_cost.argtypes = [C.c_void_p, C.POINTER(OrCost), dp]
        L.or_terrain_height.argtypes = [C.c_void_p, C.c_double, C.c_double, dp, dp, dp]
        L.or_spline_basis.argtypes = [C.c_int, C.c_int, dp]
        L.or_spline_eval.argtypes = [fp, C.c_double, dp]
        L.or_gait_ref.argtypes = [C.POINTER(OrCost), C.c_double, dp]
        L.or_gait_ref_x.argtypes = [C.POINTER(OrCost), C.c_double, dp, dp]
        L.or_ground_under.restype = C.c_double
        L.or_ground_under.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_lnf.restype = C.c_float
        L.or_lnf.argtypes = [C.c_float]
        L.or_lnf_many.argtypes = [fp, fp, C.c_long]
        L.or_sincos_u24_many.argtypes = [u32p, fp, fp, C.c_long]
        L.or_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, fp]
        L.or_noise_many.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u32p, C.c_long, fp]
        L.or_sample.argtypes = [C.POINTER(OrMppi), fp, fp, C.c_uint32, fp]
        L.or_update.restype = C.c_int
        L.or_update.argtypes = [fp, fp, C.c_int, C.c_double, fp, dp]
        L.or_update_dim.restype = C.c_int
        L.or_update_dim.argtypes = [dp, fp, C.c_int, C.c_int, C.c_double, fp, dp]
        L.or_shift_mode.argtypes = [fp, C.c_int, C.c_int, C.c_int, fp]
        L.or_controls.argtypes = [C.c_int, C.c_int, C.c_int, fp, dp]
        L.or_interp_basis.argtypes = [C.c_int, C.c_int, C.c_int, dp]
        L.or_update_d.restype = C.c_int
        L.or_update_d.argtypes = [dp, fp, C.c_int, C.c_double, fp, dp]
        L.or_shift.argtypes = [fp, C.c_int, C.c_int, fp]
        L.or_mppi_step.restype = C.c_int
        L.or_mppi_step.argtypes = [C.c_void_p, C.POINTER(OrCost), C.POINTER(OrMppi), dp, fp, fp,
                                   C.c_uint32, fp, fp, fp, C.c_int]
        L.or_dt_steps.argtypes = [C.c_void_p, dp, dp, C.c_long, C.c_int, C.c_double, dp, C.c_int]
        L.or_stage_costs.argtypes = [C.c_void_p, C.POINTER(OrCost), dp, dp, dp, C.c_long, dp]
        L.or_tree_init.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_tree_add.restype = C.c_int
        L.or_tree_add.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_double, dp, dp]
        L.or_tree_nq.restype = C.c_int
        L.or_tree_nq.argtypes = [C.c_void_p]
        L.or_tree_nv.restype = C.c_int
        L.or_tree_nv.argtypes = [C.c_void_p]
        for name in ("or_aba", "or_rnea"):
            getattr(L, name).argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp]
        L.or_crba.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_fk.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_body_vel.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_momentum_world.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_momentum_rate_world.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------- model, cost, MPPI settings ----------------

class World:
    """The oracle's world (robot tree, contact spheres, terrain, optional box)."""

    def __init__(self, robot: dict):
        L = lib()
        p = OrParams()
        keep = []
        for name, ct in OrParams._fields_:
            if name in ("hf", "sbox_lo", "sbox_hi"):
                continue
            val = robot[name]
            if isinstance(val, (tuple, list, np.ndarray)):
                arr = getattr(p, name)
                for i, v in enumerate(val):
                    arr[i] = v
            else:
                setattr(p, name, val)
        if robot.get("hf") is not None:
            hf = _f32(robot["hf"])
            keep.append(hf)
            p.hf = _p(hf, C.c_float)
        for i, (lo, hi) in enumerate(zip(robot["sbox_lo"], robot["sbox_hi"])):
            for a in range(3):
                p.sbox_lo[i][a] = lo[a]
                p.sbox_hi[i][a] = hi[a]
        self._keep = keep
        self.params = p
        self.buf = C.create_string_buffer(L.or_world_size())
        L.or_world_init(self.buf, C.byref(p))
        self.nx = 50 if robot["has_box"] else 37

    @property
    def ptr(self):
        return C.cast(self.buf, C.c_void_p)


def make_cost(cost: dict) -> OrCost:
    c = OrCost()
    for name, _ in OrCost._fields_:
        val = cost[name]
        if isinstance(val, (tuple, list, np.ndarray)):
            arr = getattr(c, name)
            for i, v in enumerate(val):
                arr[i] = v
        else:
            setattr(c, name, val)
    return c


def make_mppi(m: dict) -> OrMppi:
    o = OrMppi()
    o.K, o.H, o.n_sub, o.ctrl_steps = m["K"], m["H"], m["n_sub"], m["ctrl_steps"]
    o.dt, o.lam = m["dt"], m["lam"]
    for i in range(48):
        o.sigma[i] = float(m["sigma"][i])
    for i in range(3):
        o.q_lo[i] = float(m["q_lo"][i])
        o.q_hi[i] = float(m["q_hi"][i])
    o.seed, o.inst, o.n_prop = int(m["seed"]), int(m["inst"]), int(m.get("n_prop", 0))
    o.interp = interp_of(m)
    return o


# ---------------- dynamics of the world ----------------

def substep(world: World, x, u, h):
    x = _f64(x).copy()
    lib().or_substep(world.ptr, _p(x, C.c_double), _p(_f64(u), C.c_double), h)
    return x


def contact_fext(world: World, x):
    x = _f64(x)
    fext = np.zeros((16, 6))
    fbox = np.zeros(6)
    lib().or_contact_fext(world.ptr, _p(x, C.c_double), _p(fext, C.c_double), _p(fbox, C.c_double))
    return fext[:13], fbox


def terrain_height(world: World, x, y):
    h, hx, hy = C.c_double(), C.c_double(), C.c_double()
    lib().or_terrain_height(world.ptr, x, y, C.byref(h), C.byref(hx), C.byref(hy))
    return h.value, hx.value, hy.value


def rollout(world: World, cost: dict, H, n_sub, dt, t0, x0, U, traj=False):
    U = _f32(U)
    x0 = _f64(x0)
    tr = np.zeros((H + 1, world.nx)) if traj else None
    c = make_cost(cost)
    L = lib().or_rollout(world.ptr, C.byref(c), H, n_sub, dt, t0, _p(x0, C.c_double),
                         _p(U, C.c_float), _p(tr, C.c_double) if traj else None)
    return (L, tr) if traj else L


def rollouts(world: World, cost: dict, m: dict, t0, x0, U, traj=False, nthreads=None):
    U = _f32(U).reshape(-1, param_dim(m))
    n = U.shape[0]
    x0 = _f64(x0)
    per = 1 if x0.ndim == 2 else 0
    L = np.zeros(n)
    tr = np.zeros((n, m["H"] + 1, world.nx)) if traj else None
    nthreads = nthreads or os.cpu_count() or 1
    c, mm = make_cost(cost), make_mppi(m)
    lib().or_rollouts(world.ptr, C.byref(c), C.byref(mm), t0, _p(x0, C.c_double), per,
                      _p(U, C.c_float), n, _p(L, C.c_double),
                      _p(tr, C.c_double) if traj else None, nthreads)
    return (L, tr) if traj else L


def dt_steps(world: World, X, Ut, n_sub, h, nthreads=None):
    """One dt step (n_sub sub-steps) from each state X[m][nx] with targets Ut[m][12]."""
    X = _f64(X).reshape(-1, world.nx)
    Ut = _f64(Ut).reshape(-1, NJ)
    out = np.zeros_like(X)
    lib().or_dt_steps(world.ptr, _p(X, C.c_double), _p(Ut, C.c_double), X.shape[0], n_sub, h,
                      _p(out, C.c_double), nthreads or os.cpu_count() or 1)
    return out


def stage_costs(world: World, cost: dict, X, Ut=None, t_abs=None):
    """Stage costs of (X[m], Ut[m], t_abs[m]); terminal costs when t_abs is None."""
    X = _f64(X).reshape(-1, world.nx)
    m = X.shape[0]
    out = np.zeros(m)
    c = make_cost(cost)
    if t_abs is None:
        lib().or_stage_costs(world.ptr, C.byref(c), _p(X, C.c_double), None, None, m,
                             _p(out, C.c_double))
    else:
        Ut = _f64(Ut).reshape(-1, NJ)
        ta = _f64(t_abs).reshape(-1)
        lib().or_stage_costs(world.ptr, C.byref(c), _p(X, C.c_double), _p(Ut, C.c_double),
                             _p(ta, C.c_double), m, _p(out, C.c_double))
    return out


def stage_cost(world: World, cost: dict, x, u, t_abs):
    c = make_cost(cost)
    return lib().or_stage_cost(world.ptr, C.byref(c), _p(_f64(x), C.c_double),
                               _p(_f64(u), C.c_double), t_abs)


def gait_ref(cost: dict, t_abs):
    out = np.zeros(NJ)
    c = make_cost(cost)
    lib().or_gait_ref(C.byref(c), t_abs, _p(out, C.c_double))
    return out


# ---------------- spline ----------------

def spline_basis(H, t):
    B = np.zeros(4)
    lib().or_spline_basis(H, t, _p(B, C.c_double))
    return B


def spline_eval(U, tau):
    out = np.zeros(NJ)
    lib().or_spline_eval(_p(_f32(U), C.c_float), tau, _p(out, C.c_double))
    return out


# ---------------- sampling ----------------

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def lnf(x):
    x = _f32(x)
    y = np.empty_like(x)
    lib().or_lnf_many(_p(x, C.c_float), _p(y, C.c_float), x.size)
    return y


def sincos_u24(n):
    n = np.ascontiguousarray(n, dtype=np.uint32)
    c = np.empty(n.shape, np.float32)
    s = np.empty(n.shape, np.float32)
    lib().or_sincos_u24_many(_p(n, C.c_uint32), _p(c, C.c_float), _p(s, C.c_float), n.size)
    return c, s


def noise(seed, step, inst, ks):
    ks = np.ascontiguousarray(np.atleast_1d(ks), dtype=np.uint32)
    eps = np.zeros((ks.size, D), np.float32)
    lib().or_noise_many(seed, step, inst, _p(ks, C.c_uint32), ks.size, _p(eps, C.c_float))
    return eps


def sample(m: dict, mu, step, mu_prop=None):
    mm = make_mppi(m)
    U = np.zeros((m["K"], param_dim(m)), np.float32)
    mp = _f32(mu_prop) if mu_prop is not None else None
    lib().or_sample(C.byref(mm), _p(_f32(mu), C.c_float),
                    _p(mp, C.c_float) if mp is not None else None, step, _p(U, C.c_float))
    return U


# ---------------- update ----------------

def update(L, U, lam, double_costs=False, dim=None):
    """Eq. 1 + Eq. 2 over K samples of `dim` parameters (48 by default)."""
    dim = D if dim is None else dim
    U = _f32(U).reshape(-1, dim)
    K = U.shape[0]
    mu = np.zeros(dim, np.float32)
    w = np.zeros(K)
    if dim != D:
        rc = lib().or_update_dim(_p(_f64(L), C.c_double), _p(U, C.c_float), K, dim, lam,
                                 _p(mu, C.c_float), _p(w, C.c_double))
    elif double_costs:
        rc = lib().or_update_d(_p(_f64(L), C.c_double), _p(U, C.c_float), K, lam,
                               _p(mu, C.c_float), _p(w, C.c_double))
    else:
        rc = lib().or_update(_p(_f32(L), C.c_float), _p(U, C.c_float), K, lam,
                             _p(mu, C.c_float), _p(w, C.c_double))
    return rc, mu, w


def shift(mu, H, ctrl_steps, interp=0):
    mu = _f32(mu)
    out = np.zeros(mu.shape[0], np.float32)
    lib().or_shift_mode(_p(mu, C.c_float), INTERP[interp] if isinstance(interp, str) else int(interp),
                        H, ctrl_steps, _p(out, C.c_float))
    return out


def controls(interp, H, t, U):
    """Joint targets u_t[12] of dt step t for one sample's parameters U."""
    u = np.zeros(NJ)
    lib().or_controls(INTERP[interp] if isinstance(interp, str) else int(interp), H, t,
                      _p(_f32(U), C.c_float), _p(u, C.c_double))
    return u


def interp_basis(interp, H, t):
    B = np.zeros(4)
    lib().or_interp_basis(INTERP[interp] if isinstance(interp, str) else int(interp), H, t,
                          _p(B, C.c_double))
    return B


def mppi_step(world: World, cost: dict, m: dict, x0, mu, step, mu_prop=None, nthreads=None):
    """One control step of Alg. 1.  Returns (rc, mu_new, u0, L(float32), U)."""
    mu = _f32(mu).copy()
    u0 = np.zeros(NJ, np.float32)
    L = np.zeros(m["K"], np.float32)
    U = np.zeros((m["K"], param_dim(m)), np.float32)
    c, mm = make_cost(cost), make_mppi(m)
    mp = _f32(mu_prop) if mu_prop is not None else None
    rc = lib().or_mppi_step(world.ptr, C.byref(c), C.byref(mm), _p(_f64(x0), C.c_double),
                            _p(mu, C.c_float), _p(mp, C.c_float) if mp is not None else None,
                            step, _p(u0, C.c_float), _p(L, C.c_float), _p(U, C.c_float),
                            nthreads or os.cpu_count() or 1)
    return rc, mu, u0, L, U


# ---------------- generic trees (for the dynamics pins) ----------------

class Tree:
    def __init__(self, floating: bool, gz: float = -9.81):
        L = lib()
        self.buf = C.create_string_buffer(L.or_tree_size())
        L.or_tree_init(self.ptr, int(floating), gz)

    @property
    def ptr(self):
        return C.cast(self.buf, C.c_void_p)

    def add(self, parent, axis, xtree, mass, com, Ic):
        return lib().or_tree_add(self.ptr, parent, axis, _p(_f64(xtree), C.c_double), mass,
                                 _p(_f64(com), C.c_double),
                                 _p(_f64(np.asarray(Ic).reshape(9)), C.c_double))

    @property
    def nq(self):
        return lib().or_tree_nq(self.ptr)

    @property
    def nv(self):
        return lib().or_tree_nv(self.ptr)

    def aba(self, q, v, tau, fext=None, arm=None):
        acc = np.zeros(self.nv)
        fe = _f64(fext) if fext is not None else None
        am = _f64(arm) if arm is not None else None
        lib().or_aba(self.ptr, _p(_f64(q), C.c_double), _p(_f64(v), C.c_double),
                     _p(_f64(tau), C.c_double), _p(fe, C.c_double) if fe is not None else None,
                     _p(am, C.c_double) if am is not None else None, _p(acc, C.c_double))
        return acc

    def rnea(self, q, v, acc, fext=None, arm=None):
        tau = np.zeros(self.nv)
        fe = _f64(fext) if fext is not None else None
        am = _f64(arm) if arm is not None else None
        lib().or_rnea(self.ptr, _p(_f64(q), C.c_double), _p(_f64(v), C.c_double),
                      _p(_f64(acc), C.c_double), _p(fe, C.c_double) if fe is not None else None,
                      _p(am, C.c_double) if am is not None else None, _p(tau, C.c_double))
        return tau

    def crba(self, q, arm=None):
        M = np.zeros((self.nv, self.nv))
        am = _f64(arm) if arm is not None else None
        lib().or_crba(self.ptr, _p(_f64(q), C.c_double),
                      _p(am, C.c_double) if am is not None else None, _p(M, C.c_double))
        return M

    def fk(self, q):
        R = np.zeros((16, 3, 3))
        p = np.zeros((16, 3))
        lib().or_fk(self.ptr, _p(_f64(q), C.c_double), _p(R, C.c_double), _p(p, C.c_double))
        return R, p

    def momentum(self, q, v):
        h = np.zeros(6)
        lib().or_momentum_world(self.ptr, _p(_f64(q), C.c_double), _p(_f64(v), C.c_double),
                                _p(h, C.c_double))
        return h

    def momentum_rate(self, q, v, acc):
        h = np.zeros(6)
        lib().or_momentum_rate_world(self.ptr, _p(_f64(q), C.c_double), _p(_f64(v), C.c_double),
                                     _p(_f64(acc), C.c_double), _p(h, C.c_double))
        return h


def world_tree(world: World) -> Tree:
    """A Tree view of the world's robot tree (or_world begins with its or_tree)."""
    t = Tree.__new__(Tree)
    t.buf = world.buf
    return t


class use_float:
    """Context: the same oracle source compiled with `real` = float, as the
    reference for what plain FP32 arithmetic achieves on the same inputs (the
    "FP32 floor").  Worlds must be created inside the context."""

    def __enter__(self):
        global _lib
        self._saved = (_lib, _build.build)
        path = _build.build_variant("float")
        _lib = None
        _build.build = lambda force=False: path
        return self

    def __exit__(self, *a):
        global _lib
        _lib, _build.build = self._saved


class use_count:
    """Context: the same oracle source compiled with `real` = an operation-counting
    scalar; `opcounts()` reads (and clears) the operations performed since the
    last read.  Worlds must be created inside the context; run single-threaded."""

    def __enter__(self):
        global _lib
        self._saved = (_lib, _build.build)
        path = _build.build_count()
        _lib = None
        _build.build = lambda force=False: path
        lib().or_opcount_take.argtypes = [C.POINTER(C.c_ulonglong)]
        self.opcounts()
        return self

    def opcounts(self) -> dict:
        out = (C.c_ulonglong * 6)()
        lib().or_opcount_take(out)
        return dict(zip(("add", "mul", "div", "sqrt", "trans", "cmp"), (int(v) for v in out)))

    def __exit__(self, *a):
        global _lib
        _lib, _build.build = self._saved


def gait_ref_x(cost: dict, t_abs: float, x=None):
    """u_ref(t) with the state's feedback (gait 2 reads the trunk's v_x)."""
    u = np.zeros(NJ)
    xx = _f64(x) if x is not None else None
    lib().or_gait_ref_x(C.byref(make_cost(cost)), t_abs, _p(xx, C.c_double) if xx is not None else None,
                        _p(u, C.c_double))
    return u


def ground_under(world: World, x: float, y: float) -> float:
    """Ground height under (x, y): terrain, or a static box top whose footprint contains it."""
    return lib().or_ground_under(world.ptr, x, y)
