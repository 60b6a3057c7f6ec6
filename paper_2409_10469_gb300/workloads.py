"""Seeded synthetic inputs for the whole-body MPPI path.

This module holds input descriptions and seeded generators only: the robot's
raw physical description, cost weights, MPPI settings, start states, terrain
heightfields, multi-instance mixes and serving arrivals.  It performs none of
the method's arithmetic (no dynamics, no spline, no sampling, no update), so
that both the CUDA path and the FP64 oracle can be fed from it.

The paper (arXiv 2409.10469) runs a Unitree Go1 in MuJoCo with hyperparameters
that are not published with it (Sec. IV-A); the numbers here are the model
spec's readings: trunk 5.2 kg box 0.38 x 0.09 x 0.11 m, 4 legs of
(hip-abduction, hip-flexion, knee), thigh/calf 0.213 m with 1.0/0.2 kg, foot
spheres r = 0.02, contact k = 2e4 N/m, c = 200 N s/m, mu = 0.8, kp = 30,
kd = 1, 100 Hz control (Sec. IV-A), lambda = 0.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NJ = 12
NKNOT = 4
D = NKNOT * NJ
NQ = 19
NV = 18
NX_ROBOT = NQ + NV
NX_BOX = NX_ROBOT + 13

STAND = (0.0, 0.8, -1.6)          # (abduction, hip flexion, knee) per leg, rad
Q_LO = (-0.8, -1.0, -2.7)
Q_HI = (0.8, 3.5, -0.9)


def robot(terrain: str = "plane", box: bool = False, heightfield: np.ndarray | None = None,
          hf_cell: float = 0.02, hf_origin=(0.0, 0.0), static_boxes=(), n_sub_dt=None) -> dict:
    """Raw physical description of the quadruped, its contacts and terrain."""
    p = dict(
        trunk_mass=5.2, trunk_size=(0.38, 0.09, 0.11),
        hip_x=0.19, hip_y=0.045, hip_z=0.0,
        abd_mass=0.5, abd_radius=0.04,
        thigh_offset_y=0.08,
        thigh_mass=1.0, thigh_length=0.213,
        calf_mass=0.2, calf_length=0.213,
        rod_radius=0.02, foot_radius=0.02,
        n_trunk_spheres=3, trunk_sphere_x=(-0.15, 0.0, 0.15, 0.0), trunk_sphere_r=0.055,
        gravity=9.81,
        kp=30.0, kd=1.0, armature=0.0,
        k_contact=2.0e4, c_contact=200.0, mu=0.8, eps_v=0.3,
        has_box=int(box), box_mass=3.0, box_size=(0.5, 0.5, 0.4), box_corner_r=0.01,
        terrain=0, hf_nx=0, hf_ny=0, hf_cell=hf_cell, hf_x0=float(hf_origin[0]),
        hf_y0=float(hf_origin[1]), hf=None,
        n_static_boxes=0, sbox_lo=[], sbox_hi=[],
    )
    if terrain == "heightfield":
        assert heightfield is not None
        hf = np.ascontiguousarray(heightfield, dtype=np.float32)
        p.update(terrain=1, hf_ny=hf.shape[0], hf_nx=hf.shape[1], hf=hf)
    for lo, hi in static_boxes:
        p["sbox_lo"].append(tuple(float(v) for v in lo))
        p["sbox_hi"].append(tuple(float(v) for v in hi))
    p["n_static_boxes"] = len(p["sbox_lo"])
    return fp32_geometry(p)


# Lengths that place the contact spheres: the model's values are these decimals
# rounded to the nearest FP32 number, so that the FP32 kernels and the FP64
# oracle place every sphere, box face and terrain cell at the same point (a
# 0.213 m link differs from its FP32 value by ~5e-9 m, which the 2e4 N/m contact
# stiffness would turn into a systematic force difference).
GEOMETRY_KEYS = ("hip_x", "hip_y", "hip_z", "thigh_offset_y", "thigh_length", "calf_length", "foot_radius",
                 "trunk_sphere_x", "trunk_sphere_r", "box_size", "box_corner_r", "hf_cell", "hf_x0", "hf_y0",
                 "sbox_lo", "sbox_hi")


def _f32(v):
    if isinstance(v, (list, tuple)):
        return type(v)(_f32(x) for x in v)
    return float(np.float32(v))


def fp32_geometry(p: dict) -> dict:
    for k in GEOMETRY_KEYS:
        p[k] = _f32(p[k])
    return p


def cost(task: str = "stand", box_goal=(1.5, 0.0)) -> dict:
    """Cost weights of L_walk (+ L_box for the push task), model-spec readings."""
    c = dict(w_z=1.0e3, z_ref=0.3, w_o=1.0e2, w_v=0.0, v_ref=0.0, w_p=0.0, goal_xy=(0.0, 0.0),
             w_u=1.0, w_box=0.0, box_goal_xy=(0.0, 0.0), gait=0, gait_period=0.5,
             gait_hip_amp=0.1, gait_knee_amp=0.3, stand=STAND, w_terminal=1.0,
             raibert_k=0.0, raibert_len=0.3, z_rel=0)
    if task == "trot":
        c.update(w_v=1.0e2, v_ref=0.5, gait=1)
    elif task == "trot_raibert":
        # the trot reference with the Raibert heuristic's foot-placement feedback
        c.update(w_v=1.0e2, v_ref=0.5, gait=2, raibert_k=0.1)
    elif task == "climb":
        # the trot reference, a waypoint on top of the box, height from the ground under the trunk
        c.update(w_v=1.0e2, v_ref=0.5, gait=1, w_p=1.0e1, goal_xy=(1.1, 0.0), z_rel=1)
    elif task == "push":
        c.update(w_box=1.0e2, box_goal_xy=tuple(box_goal), w_p=1.0e1, gait=1)
    elif task != "stand":
        raise ValueError(task)
    return c


def mppi(K: int, H: int, dt: float, sigma: float, n_sub: int, lam: float = 0.1,
         ctrl_period: float = 0.01, seed: int = 0, inst: int = 0, n_prop: int = 0) -> dict:
    ctrl_steps = max(1, int(round(ctrl_period / dt)))
    return dict(K=K, H=H, n_sub=n_sub, ctrl_steps=ctrl_steps, dt=dt, lam=lam,
                sigma=np.full(D, sigma, dtype=np.float32),
                q_lo=np.array(Q_LO, np.float32), q_hi=np.array(Q_HI, np.float32),
                seed=seed, inst=inst, n_prop=n_prop)


# sub-step h = 0.625 ms (model spec): the largest h at which the explicit
# contact damping and friction slopes are inside the semi-implicit Euler
# stability limit, so that rollouts are well-conditioned
H_SUB = 0.000625


def n_sub_for(dt: float) -> int:
    return max(1, int(math.ceil(dt / H_SUB - 1e-9)))


def stand_state(z: float = 0.32, box_xy=None) -> np.ndarray:
    """Trunk level at height z, legs in the stand pose, at rest."""
    x = np.zeros(NX_ROBOT if box_xy is None else NX_BOX, dtype=np.float64)
    x[2] = z
    x[3] = 1.0
    x[7:19] = np.tile(STAND, 4)
    if box_xy is not None:
        x[37:40] = (box_xy[0], box_xy[1], 0.21)
        x[40] = 1.0
    return x


def stand_mu() -> np.ndarray:
    return np.tile(np.array(STAND, np.float32), 4 * NKNOT).astype(np.float32)


def perturbed_stand(seed: int = 1, amp: float = 0.1) -> np.ndarray:
    """Stand state with joint offsets U(-amp, amp) (numpy PCG64, seeded)."""
    rng = np.random.default_rng(seed)
    x = stand_state()
    x[7:19] += rng.uniform(-amp, amp, NJ)
    return x


def random_states(n: int, seed: int, box: bool = False, spread: float = 1.0) -> np.ndarray:
    """Diverse seeded robot states around the stand for parity tests: trunk
    tilted by up to ~0.2 rad, heights 0.25..0.36 m (some feet in contact), joint
    angles and all velocities randomised."""
    rng = np.random.default_rng(seed)
    nx = NX_BOX if box else NX_ROBOT
    X = np.zeros((n, nx))
    for i in range(n):
        x = stand_state(box_xy=(0.6, 0.0) if box else None)
        x[0:2] = rng.uniform(-0.2, 0.2, 2)
        x[2] = rng.uniform(0.25, 0.36)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = rng.uniform(0, 0.2 * spread)
        x[3] = math.cos(ang / 2)
        x[4:7] = math.sin(ang / 2) * ax
        x[7:19] += rng.uniform(-0.3, 0.3, NJ) * spread
        x[19:22] = rng.normal(0, 1.0 * spread, 3)
        x[22:25] = rng.normal(0, 0.5 * spread, 3)
        x[25:37] = rng.normal(0, 3.0 * spread, NJ)
        if box:
            x[37:39] = (0.45 + rng.uniform(-0.05, 0.05), rng.uniform(-0.1, 0.1))
            x[39] = 0.2 + rng.uniform(-0.01, 0.01)
            x[44:50] = rng.normal(0, 0.2, 6)
        X[i] = x
    return X


def heightfield(seed: int = 3, n: int = 128, n_bumps: int = 20, cell: float = 0.02,
                amp: float = 0.1) -> np.ndarray:
    """n x n heights at `cell` spacing: a sum of seeded Gaussians, centres
    U(0, n*cell)^2, widths U(0.1, 0.4) m, amplitudes U(-1, 1), rescaled so
    that max |h| = amp."""
    rng = np.random.default_rng(seed)
    xs = np.arange(n) * cell
    X, Y = np.meshgrid(xs, xs)  # [y][x]
    h = np.zeros((n, n))
    for _ in range(n_bumps):
        cx, cy = rng.uniform(0, n * cell, 2)
        s = rng.uniform(0.1, 0.4)
        a = rng.uniform(-1, 1)
        h += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * s * s))
    h *= amp / np.max(np.abs(h))
    return h.astype(np.float32)


@dataclass
class Workload:
    name: str
    robot: dict
    cost: dict
    mppi: dict
    x0: np.ndarray
    mu0: np.ndarray
    steps: int = 1
    extra: dict = field(default_factory=dict)


def config_stand(K: int = 64, H: int = 50) -> Workload:
    """Plain MPPI, stand on a flat plane: dt 0.01, H 50, sigma 0.2, K 64, 10 steps."""
    dt = 0.01
    return Workload("stand_flat_K%d_H%d" % (K, H), robot(), cost("stand"),
                    mppi(K, H, dt, 0.2, n_sub_for(dt), seed=0), stand_state(), stand_mu(), 10)


def config_trot(K: int = 1024, H: int = 100) -> Workload:
    """Plain MPPI trot, flat plane: dt 0.005, H 100, sigma 0.3, v_ref 0.5 m/s,
    200 control steps from a perturbed stand."""
    dt = 0.005
    return Workload("trot_flat_K%d_H%d" % (K, H), robot(), cost("trot"),
                    mppi(K, H, dt, 0.3, n_sub_for(dt), seed=0), perturbed_stand(1), stand_mu(), 200)


def config_trot_raibert(K: int = 1024, H: int = 100) -> Workload:
    """The trot task with the Raibert-feedback gait reference."""
    dt = 0.005
    return Workload("trot_raibert_K%d_H%d" % (K, H), robot(), cost("trot_raibert"),
                    mppi(K, H, dt, 0.3, n_sub_for(dt), seed=0), perturbed_stand(1), stand_mu(), 200)


def config_terrain(K: int = 1024, H: int = 100, seed: int = 3) -> Workload:
    """Trot over a 128 x 128 heightfield (2 cm cells) plus a 0.3 m step-up box."""
    dt = 0.005
    hf = heightfield(seed)
    rb = robot("heightfield", heightfield=hf, hf_origin=(-1.28, -1.28),
               static_boxes=[((0.8, -0.5, -0.2), (1.4, 0.5, 0.3))])
    return Workload("trot_terrain_K%d_H%d" % (K, H), rb, cost("trot"),
                    mppi(K, H, dt, 0.3, n_sub_for(dt), seed=0), stand_state(z=0.42), stand_mu(), 50)


def config_climb(K: int = 1024, H: int = 100, box_height: float = 0.24, gait: str = "climb") -> Workload:
    """Climb onto a box (Sec. IV-C: up to 0.24 m, about the standing height):
    flat plane, static box from x = 0.45 m to 1.65 m (1.2 m wide) of the given
    height, waypoint at x = 1.1 m on top of it; trot reference; the height
    reference is measured from the ground under the trunk."""
    dt = 0.005
    rb = robot(static_boxes=[((0.45, -0.6, -0.2), (1.65, 0.6, box_height))])
    return Workload("climb_%02dcm_K%d_H%d" % (round(100 * box_height), K, H), rb, cost(gait),
                    mppi(K, H, dt, 0.3, n_sub_for(dt), seed=0), perturbed_stand(1), stand_mu(), 400)


def config_push(K: int = 4096, H: int = 100, seed: int = 100, n_prop: int = 0) -> Workload:
    """Box pushing: free 0.5 x 0.5 x 0.4 m, 3 kg box whose centre starts 0.5 m
    ahead of the trunk (near face 0.25 m ahead, within reach); box goal offset
    U(0.5, 1.5) m further forward; the robot's position goal is the box's start
    centre."""
    rng = np.random.default_rng(seed)
    dt = 0.005
    bx = 0.5
    goal = (bx + rng.uniform(0.5, 1.5), 0.0)
    c = cost("push", box_goal=goal)
    c["goal_xy"] = (bx, 0.0)
    return Workload("push_K%d_H%d" % (K, H), robot(box=True), c,
                    mppi(K, H, dt, 0.3, n_sub_for(dt), seed=0, n_prop=n_prop),
                    stand_state(box_xy=(bx, 0.0)), stand_mu(), 100, dict(goal=goal))


def multi_instance_mix(n: int = 16, seed: int = 2):
    """(K, H) of n instances: K from {256..4096}, H from {50, 100, 150}."""
    rng = np.random.default_rng(seed)
    Ks = rng.choice([256, 512, 1024, 2048, 4096], n)
    Hs = rng.choice([50, 100, 150], n)
    return [(int(k), int(h)) for k, h in zip(Ks, Hs)]


def serving_robots(n_robots: int = 64, seed: int = 4, K_range=(512, 8192), H_range=(50, 150)):
    """Per-robot (task, K, H) of the serving workload: tasks cycle through
    stand / trot / terrain / push, K ~ U{512..8192}, H ~ U{50..150}."""
    rng = np.random.default_rng(seed)
    tasks = ["stand", "trot", "terrain", "push"]
    return [(tasks[r % len(tasks)], int(rng.integers(K_range[0], K_range[1] + 1)),
             int(rng.integers(H_range[0], H_range[1] + 1))) for r in range(n_robots)]


def serving_arrivals(n_robots: int = 64, rate_hz: float = 50.0, duration: float = 1.0,
                     seed: int = 4):
    """Poisson request times of every robot over `duration` seconds:
    sorted list of (t, robot)."""
    rng = np.random.default_rng(seed + 1000)
    out = []
    for r in range(n_robots):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration:
            out.append((t, r))
            t += rng.exponential(1.0 / rate_hz)
    out.sort()
    return out


def task_config(task: str, K: int, H: int) -> "Workload":
    return {"stand": config_stand, "trot": config_trot, "terrain": config_terrain,
            "push": config_push}[task](K=K, H=H)


MLP_SIZES = [(256, 62), (256, 256), (256, 256), (48, 256)]


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the proposal network (flat FP32, layout
    W1 [256][62], b1, W2, b2, W3, b3, W4 [48][256], b4): weights uniform in
    +-sqrt(6 / (fan_in + fan_out)), biases zero."""
    rng = np.random.default_rng(seed)
    out = []
    for no, ni in MLP_SIZES:
        lim = math.sqrt(6.0 / (ni + no))
        out.append(rng.uniform(-lim, lim, no * ni))
        out.append(np.zeros(no))
    return np.concatenate(out).astype(np.float32)
