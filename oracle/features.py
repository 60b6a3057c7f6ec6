"""FP64 oracle of the proposal network's 62 input features (TEST
INFRASTRUCTURE ONLY); the definition is the model spec's (see the CUDA
kernel's header in the library for the same list)."""
from __future__ import annotations

import math

import numpy as np


def features(x, cost: dict, ctrl_steps: int, dt: float, step: int) -> np.ndarray:
    x = np.asarray(x, np.float64)
    f = np.zeros(62)
    f[0] = x[2]
    sq = -1.0 if x[3] < 0 else 1.0
    f[1:5] = sq * x[3:7]
    f[5:17] = x[7:19]
    f[17:23] = x[19:25]
    f[23:35] = 0.1 * x[25:37]
    box = x.size >= 50
    if box:
        f[35:37] = x[37:39] - x[0:2]
        f[37] = x[39]
        sb = -1.0 if x[40] < 0 else 1.0
        f[38:42] = sb * x[40:44]
        f[42:48] = x[44:50]
        f[48:50] = np.asarray(cost["box_goal_xy"]) - x[37:39]
    f[50:52] = np.asarray(cost["goal_xy"]) - x[0:2]
    phase = 0.0
    if cost["gait"] in (1, 2) and cost["gait_period"] > 0:
        t = step * ctrl_steps * dt
        phase = 2 * math.pi * math.fmod(t, cost["gait_period"]) / cost["gait_period"]
    f[52], f[53] = math.sin(phase), math.cos(phase)
    w, qx, qy, qz = x[3:7]
    f[54:57] = (2 * (qx * qz - w * qy), 2 * (qy * qz + w * qx), 1 - 2 * (qx * qx + qy * qy))
    if box:
        bw, bx, by, bz = x[40:44]
        f[57:59] = (1 - 2 * (by * by + bz * bz), 2 * (bx * by + bw * bz))
        f[59] = math.hypot(f[48], f[49])
        f[60] = math.hypot(f[35], f[36])
    f[61] = 1.0
    return f
