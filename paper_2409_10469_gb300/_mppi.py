"""Thin ctypes binding of the C ABI in include/mppi.h (libmppi_gb300.so).

Argument marshalling only: every step of the MPPI path (sampling, rollouts,
update, shift) runs in the library's CUDA kernels.  Buffers may be torch
tensors (device or host) or numpy arrays; they are passed as raw pointers.
The library must be built (``paper_2409_10469_gb300.build``); importing this
module without it raises, there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmppi_gb300.so")

MPPI_OK, MPPI_ERR_ARG, MPPI_ERR_OOM, MPPI_ERR_CUDA = 0, 1, 2, 3
MPPI_ERR_NONFINITE, MPPI_ERR_TIMEOUT, MPPI_ERR_BUSY, MPPI_ERR_NOTSUP = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NONFINITE",
                5: "ERR_TIMEOUT", 6: "ERR_BUSY", 7: "ERR_NOTSUP"}

# every entry point declared in include/mppi.h
EXPORTS = ("mppi_create", "mppi_destroy", "mppi_last_error", "mppi_set_nominal",
           "mppi_get_nominal", "mppi_sample", "mppi_rollouts", "mppi_update", "mppi_step",
           "mppi_set_timing", "mppi_get_timings", "mppi_launch_count", "mppi_state_size",
           "mppi_update_noalloc", "mppi_get_samples", "mppi_step_partial", "mppi_step_finalize",
           "mppi_batch_create", "mppi_batch_destroy",
           "mppi_batch_last_error", "mppi_batch_step", "mppi_batch_set_shape", "mppi_batch_get_shape",
           "mppi_batch_autotune", "mppi_batch_launch_count", "mppi_batch_shared_model", "mppi_server_create",
           "mppi_server_destroy", "mppi_server_last_error", "mppi_server_add_robot", "mppi_server_submit",
           "mppi_server_tick", "mppi_server_poll", "mppi_server_stats", "mppi_server_reset_stats",
           "mppi_server_drain", "mppi_mlp_create", "mppi_mlp_destroy", "mppi_mlp_last_error",
           "mppi_mlp_param_count", "mppi_mlp_set_params", "mppi_mlp_get_params", "mppi_mlp_forward",
           "mppi_mlp_train_step", "mppi_tc_gemm_bf16", "mppi_features", "mppi_set_proposal", "mppi_step_proposal",
           "mppi_batch_get_means", "mppi_selftest_wait_timeout", "mppi_param_dim",
           "mppi_selftest_noise_tables")

# a shard's partial sums of a sharded step: m, Z, S[48] (MPPI_SHARD_PARTIAL)
SHARD_PARTIAL = 50

# control representations (MPPI_INTERP_* of include/mppi.h; Sec. III-B, Fig. 5)
INTERP = {"cubic": 0, "zero": 1, "linear": 2, "direct": 3}


def interp_code(v) -> int:
    return INTERP[v] if isinstance(v, str) else int(v)


class MppiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class MppiModel(C.Structure):
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
        ("hf", C.c_void_p),
        ("n_static_boxes", C.c_int), ("sbox_lo", (C.c_double * 3) * 4),
        ("sbox_hi", (C.c_double * 3) * 4),
    ]


class MppiCost(C.Structure):
    _fields_ = [
        ("w_z", C.c_double), ("z_ref", C.c_double), ("w_o", C.c_double),
        ("w_v", C.c_double), ("v_ref", C.c_double), ("w_p", C.c_double),
        ("goal_xy", C.c_double * 2), ("w_u", C.c_double), ("w_box", C.c_double),
        ("box_goal_xy", C.c_double * 2),
        ("gait", C.c_int), ("gait_period", C.c_double), ("gait_hip_amp", C.c_double),
        ("gait_knee_amp", C.c_double), ("stand", C.c_double * 3), ("w_terminal", C.c_double),
        ("raibert_k", C.c_double), ("raibert_len", C.c_double), ("z_rel", C.c_int),
    ]


class MppiConfig(C.Structure):
    _fields_ = [
        ("K", C.c_int), ("H", C.c_int), ("n_sub", C.c_int), ("ctrl_steps", C.c_int),
        ("dt", C.c_double), ("lam", C.c_double),
        ("sigma", C.c_float * 48), ("q_lo", C.c_float * 3), ("q_hi", C.c_float * 3),
        ("seed", C.c_uint64), ("inst", C.c_uint32), ("n_prop", C.c_int), ("block", C.c_int),
        ("interp", C.c_int),
    ]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "launches", "busy_rejects", "queued",
                                          "in_flight", "pool_bytes", "pool_in_use", "pool_peak")] + \
               [(n, C.c_double) for n in ("rollout_steps", "latency_p50", "latency_p99", "latency_max")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmppi_gb300.so is not built: run __graft_entry__.build() "
                              "(the CUDA path has no fallback)")
        L = C.CDLL(LIB_PATH)
        vp, fp = C.c_void_p, C.c_void_p
        L.mppi_create.argtypes = [C.POINTER(MppiModel), C.POINTER(MppiCost), C.POINTER(MppiConfig),
                                  vp, C.POINTER(C.c_void_p)]
        L.mppi_destroy.argtypes = [vp]
        L.mppi_last_error.restype = C.c_char_p
        L.mppi_last_error.argtypes = [vp]
        L.mppi_set_nominal.argtypes = [vp, fp]
        L.mppi_get_nominal.argtypes = [vp, fp]
        L.mppi_sample.argtypes = [vp, C.c_uint32, fp, fp]
        L.mppi_rollouts.argtypes = [vp, fp, C.c_int, fp, C.c_int, C.c_double, fp, fp]
        L.mppi_update.argtypes = [vp, fp, fp, C.c_int, fp, fp]
        L.mppi_step.argtypes = [vp, fp, C.c_uint32, fp, fp]
        L.mppi_set_timing.argtypes = [vp, C.c_int]
        L.mppi_get_timings.argtypes = [vp, C.POINTER(C.c_float)]
        L.mppi_launch_count.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.mppi_get_samples.argtypes = [vp, fp, fp]
        L.mppi_step_partial.argtypes = [vp, fp, C.c_uint32, C.c_int, C.c_int, vp]
        L.mppi_step_finalize.argtypes = [vp, vp, fp, fp]
        L.mppi_update_noalloc.argtypes = [fp, fp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, fp, fp,
                                           fp, fp, fp, vp]
        L.mppi_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, vp, C.POINTER(C.c_void_p)]
        L.mppi_batch_destroy.argtypes = [vp]
        L.mppi_batch_last_error.argtypes = [vp]
        L.mppi_batch_last_error.restype = C.c_char_p
        L.mppi_batch_step.argtypes = [vp, vp, vp, vp, vp]
        L.mppi_batch_set_shape.argtypes = [vp, C.c_int, C.c_int]
        L.mppi_batch_get_shape.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.mppi_batch_autotune.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_float)]
        L.mppi_batch_launch_count.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.mppi_batch_shared_model.argtypes = [vp, C.POINTER(C.c_int)]
        L.mppi_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.mppi_server_destroy.argtypes = [vp]
        L.mppi_server_last_error.argtypes = [vp]
        L.mppi_server_last_error.restype = C.c_char_p
        L.mppi_server_add_robot.argtypes = [vp, vp, C.POINTER(C.c_int)]
        L.mppi_server_submit.argtypes = [vp, C.c_int, vp, C.c_uint32]
        L.mppi_server_tick.argtypes = [vp, C.POINTER(C.c_int)]
        L.mppi_server_poll.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.mppi_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.mppi_server_reset_stats.argtypes = [vp]
        L.mppi_server_drain.argtypes = [vp]
        L.mppi_mlp_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
        L.mppi_mlp_destroy.argtypes = [vp]
        L.mppi_mlp_last_error.argtypes = [vp]
        L.mppi_mlp_last_error.restype = C.c_char_p
        L.mppi_mlp_param_count.argtypes = [vp]
        L.mppi_mlp_param_count.restype = C.c_long
        L.mppi_mlp_set_params.argtypes = [vp, vp, vp]
        L.mppi_mlp_get_params.argtypes = [vp, vp, vp]
        L.mppi_mlp_forward.argtypes = [vp, vp, C.c_int, vp, vp]
        L.mppi_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, C.c_float, vp, vp, vp]
        L.mppi_step_proposal.argtypes = [vp, vp, vp, C.c_uint32, vp, vp]
        L.mppi_tc_gemm_bf16.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, vp]
        L.mppi_features.argtypes = [vp, vp, C.c_int, C.c_uint32, vp]
        L.mppi_batch_get_means.argtypes = [vp, vp, vp]
        L.mppi_selftest_wait_timeout.argtypes = [vp]
        L.mppi_selftest_noise_tables.argtypes = [vp, vp, vp, vp]
        L.mppi_set_proposal.argtypes = [vp, vp]
        L.mppi_state_size.argtypes = [vp]
        L.mppi_state_size.restype = C.c_int
        L.mppi_param_dim.argtypes = [vp]
        L.mppi_param_dim.restype = C.c_int
        for name in EXPORTS:
            if name not in ("mppi_last_error", "mppi_state_size", "mppi_param_dim", "mppi_batch_last_error",
                            "mppi_server_last_error", "mppi_mlp_last_error", "mppi_mlp_param_count"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a float32/uint buffer (torch tensor or numpy array), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "buffer must be contiguous"
        return C.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "buffer must be contiguous"
        return C.c_void_p(x.data_ptr())
    raise TypeError("unsupported buffer type %r" % type(x))


def _fill(struct, d: dict, skip=()):
    for name, ct in struct._fields_:
        if name in skip or name not in d:
            continue
        v = d[name]
        if isinstance(v, (tuple, list, np.ndarray)):
            arr = getattr(struct, name)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(struct, name, v)


def model_struct(robot: dict):
    m = MppiModel()
    _fill(m, robot, skip=("hf", "sbox_lo", "sbox_hi"))
    keep = None
    if robot.get("hf") is not None:
        keep = np.ascontiguousarray(robot["hf"], dtype=np.float32)
        m.hf = keep.ctypes.data
    for i, (lo, hi) in enumerate(zip(robot.get("sbox_lo", []), robot.get("sbox_hi", []))):
        for a in range(3):
            m.sbox_lo[i][a] = lo[a]
            m.sbox_hi[i][a] = hi[a]
    return m, keep


def cost_struct(cost: dict):
    c = MppiCost()
    _fill(c, cost)
    return c


def config_struct(mp: dict, block: int = 0):
    c = MppiConfig()
    c.K, c.H, c.n_sub, c.ctrl_steps = mp["K"], mp["H"], mp["n_sub"], mp["ctrl_steps"]
    c.dt, c.lam = mp["dt"], mp["lam"]
    for i in range(48):
        c.sigma[i] = float(mp["sigma"][i])
    for i in range(3):
        c.q_lo[i] = float(mp["q_lo"][i])
        c.q_hi[i] = float(mp["q_hi"][i])
    c.seed, c.inst, c.n_prop = int(mp["seed"]), int(mp["inst"]), int(mp.get("n_prop", 0))
    c.block = int(block or mp.get("block", 0))
    c.interp = interp_code(mp.get("interp", 0))
    return c


def update_noalloc(L, U, n, H, ctrl_steps, lam, mu_in, mu_out, u0_out, mu_upd_out=None,
                   status_out=None, stream=None, interp="cubic"):
    """mppi_update_noalloc: the update without a handle or any allocation (for
    callers that cannot allocate device memory); all buffers are device memory
    of the current device; interp names the knot representation."""
    return lib().mppi_update_noalloc(_ptr(L), _ptr(U), n, H, ctrl_steps, lam, interp_code(interp),
                                     _ptr(mu_in), _ptr(mu_out), _ptr(mu_upd_out), _ptr(u0_out),
                                     _ptr(status_out), stream)


class Controller:
    """One MPPI controller instance (a handle of the C ABI)."""

    def __init__(self, robot: dict, cost: dict, mppi: dict, stream=None, block: int = 0):
        L = lib()
        self._model, self._hf = model_struct(robot)
        self._cost = cost_struct(cost)
        self._cfg = config_struct(mppi, block)
        h = C.c_void_p()
        st = C.c_void_p(stream) if isinstance(stream, int) else stream
        rc = L.mppi_create(C.byref(self._model), C.byref(self._cost), C.byref(self._cfg), st,
                           C.byref(h))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_create failed")
        self.h = h
        self.K = mppi["K"]
        self.H = mppi["H"]
        self.lam = float(mppi["lam"])
        self.nx = L.mppi_state_size(h)
        self.D = L.mppi_param_dim(h)   # parameters per sample: 48, or 12 H (direct)

    def _check(self, rc):
        if rc != MPPI_OK:
            raise MppiError(rc, lib().mppi_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nominal(self, mu):
        self._check(lib().mppi_set_nominal(self.h, _ptr(mu)))

    def get_nominal(self, out=None):
        out = np.zeros(self.D, np.float32) if out is None else out
        self._check(lib().mppi_get_nominal(self.h, _ptr(out)))
        return out

    def step_partial(self, x0, step, k0, n, out=None):
        """mppi_step_partial: samples k0 .. k0 + n - 1 of control step `step`
        rolled out; returns (m, Z, S[48]) as float64[50] (host unless `out`)."""
        out = np.zeros(SHARD_PARTIAL, np.float64) if out is None else out
        self._check(lib().mppi_step_partial(self.h, _ptr(x0), int(step), int(k0), int(n), _ptr(out)))
        return out

    def step_finalize(self, sums, u0_out=None, mu_out=None, check=True):
        """mppi_step_finalize from the combined sums (Z, S[48]) of every shard."""
        sums = np.ascontiguousarray(sums, np.float64) if isinstance(sums, np.ndarray) else sums
        rc = lib().mppi_step_finalize(self.h, _ptr(sums), _ptr(u0_out), _ptr(mu_out))
        return self._check(rc) if check else rc

    def last_samples(self):
        """(U [K][D], L [K]) of the last control step (host copies)."""
        U = np.zeros((self.K, self.D), np.float32)
        L = np.zeros(self.K, np.float32)
        self._check(lib().mppi_get_samples(self.h, _ptr(U), _ptr(L)))
        return U, L

    def sample(self, step, mu_prop=None, out=None):
        self._check(lib().mppi_sample(self.h, step, _ptr(mu_prop), _ptr(out)))
        return out

    def rollouts(self, x0, U=None, n=None, t0=0.0, L_out=None, traj_out=None,
                 x0_per_sample=False):
        n = self.K if n is None else n
        self._check(lib().mppi_rollouts(self.h, _ptr(x0), int(bool(x0_per_sample)), _ptr(U), n,
                                        float(t0), _ptr(L_out), _ptr(traj_out)))
        return L_out

    def update(self, L=None, U=None, n=None, mu_out=None, u0_out=None):
        n = self.K if n is None else n
        rc = lib().mppi_update(self.h, _ptr(L), _ptr(U), n, _ptr(mu_out), _ptr(u0_out))
        if rc != MPPI_ERR_NONFINITE:
            self._check(rc)
        return rc

    def step(self, x0, step, u0_out=None, mu_out=None, check=True):
        rc = lib().mppi_step(self.h, _ptr(x0), step, _ptr(u0_out), _ptr(mu_out))
        if check and rc != MPPI_ERR_NONFINITE:
            self._check(rc)
        return rc

    def features(self, X, step, out=None):
        X = np.ascontiguousarray(X, np.float32) if isinstance(X, np.ndarray) else X
        n = X.shape[0] if X.ndim == 2 else 1
        out = np.zeros((n, 62), np.float32) if out is None else out
        self._check(lib().mppi_features(self.h, _ptr(X), n, step, _ptr(out)))
        return out

    def step_proposal(self, net, x0, step, u0_out=None, mu_out=None, check=True):
        """the learned-proposal step in one call (mppi_step_proposal): features,
        the network's forward, the proposal, the control step"""
        rc = lib().mppi_step_proposal(self.h, net.n, _ptr(x0), step, _ptr(u0_out), _ptr(mu_out))
        if check and rc != MPPI_ERR_NONFINITE:
            self._check(rc)
        return rc

    def set_proposal(self, mu_prop):
        if mu_prop is not None and isinstance(mu_prop, np.ndarray):
            mu_prop = np.ascontiguousarray(mu_prop, np.float32)
        self._check(lib().mppi_set_proposal(self.h, _ptr(mu_prop)))

    def set_timing(self, on=True):
        self._check(lib().mppi_set_timing(self.h, int(on)))

    def timings(self):
        ms = (C.c_float * 3)()
        self._check(lib().mppi_get_timings(self.h, ms))
        return list(ms)

    def launch_count(self):
        c = C.c_uint64()
        self._check(lib().mppi_launch_count(self.h, C.byref(c)))
        return c.value


class Batch:
    """Many controllers stepped by one persistent launch per control step."""

    def __init__(self, controllers, stream=None):
        L = lib()
        self.ctls = list(controllers)
        arr = (C.c_void_p * len(self.ctls))(*[c.h.value for c in self.ctls])
        b = C.c_void_p()
        st = C.c_void_p(stream) if isinstance(stream, int) else stream
        rc = L.mppi_batch_create(arr, len(self.ctls), st, C.byref(b))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_batch_create failed")
        self.b = b
        self.n = len(self.ctls)

    def _check(self, rc):
        if rc != MPPI_OK:
            raise MppiError(rc, lib().mppi_batch_last_error(self.b).decode())

    def close(self):
        if getattr(self, "b", None):
            lib().mppi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, x0s, steps, u0s=None, active=None):
        st = np.ascontiguousarray(steps, dtype=np.uint32)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
        self._check(lib().mppi_batch_step(self.b, _ptr(act), _ptr(x0s), _ptr(st), _ptr(u0s)))
        return u0s

    def set_shape(self, block, blocks_per_sm):
        self._check(lib().mppi_batch_set_shape(self.b, block, blocks_per_sm))

    def shape(self):
        b, p = C.c_int(), C.c_int()
        self._check(lib().mppi_batch_get_shape(self.b, C.byref(b), C.byref(p)))
        return b.value, p.value

    def autotune(self, x0s, trials=3):
        b, p, ms = C.c_int(), C.c_int(), C.c_float()
        self._check(lib().mppi_batch_autotune(self.b, _ptr(x0s), trials, C.byref(b), C.byref(p), C.byref(ms)))
        return b.value, p.value, ms.value

    def launch_count(self):
        c = C.c_uint64()
        self._check(lib().mppi_batch_launch_count(self.b, C.byref(c)))
        return c.value

    def shared_model(self):
        """True when all instances share one model and cost (parameter-bank kernel)"""
        c = C.c_int()
        self._check(lib().mppi_batch_shared_model(self.b, C.byref(c)))
        return bool(c.value)

    def means(self, mu_upds=None, nominals=None):
        self._check(lib().mppi_batch_get_means(self.b, _ptr(mu_upds), _ptr(nominals)))
        return mu_upds, nominals


class Server:
    """Continuous-batching serving runtime (mppi_server_*)."""

    def __init__(self, budget_bytes: int, max_robots: int, max_samples: int):
        s = C.c_void_p()
        rc = lib().mppi_server_create(budget_bytes, max_robots, max_samples, C.byref(s))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_server_create failed")
        self.s = s
        self.robots = []

    def _check(self, rc, ok=(MPPI_OK,)):
        if rc not in ok:
            raise MppiError(rc, lib().mppi_server_last_error(self.s).decode())
        return rc

    def close(self):
        if getattr(self, "s", None):
            lib().mppi_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_robot(self, ctl: "Controller") -> int:
        rid = C.c_int()
        self._check(lib().mppi_server_add_robot(self.s, ctl.h, C.byref(rid)))
        self.robots.append(ctl)
        return rid.value

    def submit(self, robot: int, x0, step: int) -> int:
        x = np.ascontiguousarray(x0, dtype=np.float32)
        return self._check(lib().mppi_server_submit(self.s, robot, _ptr(x), step),
                           ok=(MPPI_OK, MPPI_ERR_BUSY))

    def tick(self) -> int:
        n = C.c_int()
        self._check(lib().mppi_server_tick(self.s, C.byref(n)))
        return n.value

    def poll(self, robot: int):
        u0 = np.zeros(12, np.float32)
        lat, ready = C.c_double(), C.c_int()
        self._check(lib().mppi_server_poll(self.s, robot, _ptr(u0), C.byref(lat), C.byref(ready)))
        return (u0, lat.value) if ready.value else None

    def stats(self) -> dict:
        st = ServerStats()
        self._check(lib().mppi_server_stats(self.s, C.byref(st)))
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def reset_stats(self):
        self._check(lib().mppi_server_reset_stats(self.s))

    def drain(self):
        self._check(lib().mppi_server_drain(self.s))


class MLP:
    """The proposal network (mppi_mlp_*): BF16 tcgen05 forward / backward, AdamW."""

    IN, HID, OUT = 62, 256, 48

    def __init__(self, max_batch: int, stream=None):
        n = C.c_void_p()
        rc = lib().mppi_mlp_create(max_batch, C.byref(n))
        if rc != MPPI_OK:
            raise MppiError(rc, "mppi_mlp_create failed")
        self.n = n
        self.stream = C.c_void_p(stream) if isinstance(stream, int) else stream
        self.nparam = lib().mppi_mlp_param_count(n)

    def _check(self, rc):
        if rc != MPPI_OK:
            raise MppiError(rc, lib().mppi_mlp_last_error(self.n).decode())

    def close(self):
        if getattr(self, "n", None):
            lib().mppi_mlp_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        self._check(lib().mppi_mlp_set_params(self.n, _ptr(np.ascontiguousarray(p, np.float32)
                                                          if isinstance(p, np.ndarray) else p), self.stream))

    def get_params(self):
        out = np.zeros(self.nparam, np.float32)
        self._check(lib().mppi_mlp_get_params(self.n, _ptr(out), self.stream))
        return out

    def forward(self, X, out=None):
        X = np.ascontiguousarray(X, np.float32) if isinstance(X, np.ndarray) else X
        B = X.shape[0]
        out = np.zeros((B, self.OUT), np.float32) if out is None else out
        self._check(lib().mppi_mlp_forward(self.n, _ptr(X), B, _ptr(out), self.stream))
        return out

    def train_step(self, X, T, lr=1e-3, weight_decay=0.0, grad=False):
        X = np.ascontiguousarray(X, np.float32) if isinstance(X, np.ndarray) else X
        T = np.ascontiguousarray(T, np.float32) if isinstance(T, np.ndarray) else T
        loss = np.zeros(1, np.float32)
        g = np.zeros(self.nparam, np.float32) if grad else None
        self._check(lib().mppi_mlp_train_step(self.n, _ptr(X), _ptr(T), X.shape[0], lr, weight_decay,
                                              _ptr(loss), _ptr(g), self.stream))
        return (float(loss[0]), g) if grad else float(loss[0])


def tc_gemm_bf16(A_bits, B_bits, M, N, K, D):
    """D = A B^T on the tensor cores; A_bits, B_bits: device uint16 (BF16 bits)."""
    return lib().mppi_tc_gemm_bf16(_ptr(A_bits), _ptr(B_bits), _ptr(D), M, N, K, None)
