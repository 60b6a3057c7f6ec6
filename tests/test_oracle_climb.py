"""Pins of the Raibert-feedback gait reference (Sec. IV-B) and of the ground-
relative height cost used for climbing (Sec. IV-C), against what their
definitions fix."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W


def state_with_vx(vx):
    x = W.config_trot().x0.astype(np.float64).copy()
    x[22] = vx
    return x


# The reading of the Raibert-feedback reference: a swinging foot is placed
# dx = (T_stance / 2) v_x + k (v_x - v_ref) ahead of its hip, T_stance half of the
# gait period P = 0.5 s, k = 0.1 s, v_ref = 0.5 m/s, realised as the hip-flexion
# change -dx / L (L = 0.3 m) clamped to +-0.4 rad.  Written out:
#   v_x = 0.5 (= v_ref): dx = 0.125 * 0.5           = 0.0625  -> -0.208333... rad
#   v_x = 0.0:           dx = 0.1 * (0 - 0.5)       = -0.05   -> +0.166666... rad
#   v_x = -0.3:          dx = -0.0375 + 0.1 * -0.8  = -0.1175 -> +0.391666... rad
#   v_x = 1.2:           dx = 0.15 + 0.1 * 0.7      = 0.22    -> -0.7333 -> clamped -0.4
#   v_x = 5.0:           dx = 0.625 + 0.45          = 1.075   -> clamped -0.4
DTH = {0.5: -0.0625 / 0.3, 0.0: 0.05 / 0.3, -0.3: 0.1175 / 0.3, 1.2: -0.4, 5.0: -0.4}


@pytest.mark.parametrize("vx", sorted(DTH))
def test_raibert_reference_written_out(vx):
    """the stand pose (0, 0.8, -1.6), hip amplitude 0.1 and knee amplitude 0.3:
    at a quarter period (t = 0.125 s) legs FR and RL swing fully (sin = 1) --
    hip 0.9 + dth, knee -1.9 -- and FL, RR stand (sin = -1) -- hip 0.7, knee
    -1.6, no feedback; at three quarters the pairs swap; at t = 0 no leg swings
    and the reference is the stand pose whatever v_x"""
    c = W.cost("trot_raibert")
    assert (c["gait_period"], c["raibert_k"], c["raibert_len"], c["v_ref"]) == (0.5, 0.1, 0.3, 0.5)
    d = DTH[vx]
    swing, stance = [0.0, 0.9 + d, -1.9], [0.0, 0.7, -1.6]
    u = O.gait_ref_x(c, 0.125, state_with_vx(vx))
    assert u == pytest.approx(swing + stance + stance + swing, abs=1e-12)
    u = O.gait_ref_x(c, 0.375, state_with_vx(vx))
    assert u == pytest.approx(stance + swing + swing + stance, abs=1e-12)
    u = O.gait_ref_x(c, 0.0, state_with_vx(vx))
    assert u == pytest.approx([0.0, 0.8, -1.6] * 4, abs=1e-12)


def test_raibert_feedback_direction_and_clamp():
    c = W.cost("trot_raibert")
    t = 0.06                                   # legs 0 and 3 swing
    hip = lambda v: O.gait_ref_x(c, t, state_with_vx(v))[1]
    # faster than the reference: the foot goes further forward, the hip target further back
    assert hip(0.8) < hip(0.5) < hip(0.2)
    assert hip(50.0) == hip(60.0) and hip(-50.0) == hip(-60.0)   # clamped at 0.4 rad
    assert abs(hip(50.0) - hip(-50.0)) == pytest.approx(0.8 * max(0, math.sin(2 * math.pi * t / 0.5)))
    # without a state the reference velocity is used
    assert np.array_equal(O.gait_ref_x(c, t), O.gait_ref_x(c, t, state_with_vx(c["v_ref"])))


def test_ground_under_plane_boxes_and_heightfield():
    cfg = W.config_climb(K=1, H=2)
    w = O.World(cfg.robot)
    assert O.ground_under(w, 0.0, 0.0) == 0.0
    assert O.ground_under(w, 1.0, 0.3) == pytest.approx(0.24)
    assert O.ground_under(w, 1.0, 0.7) == 0.0          # beside the box
    assert O.ground_under(w, 1.7, 0.0) == 0.0          # past it
    t = W.config_terrain(K=1, H=2)
    wt = O.World(t.robot)
    h, _, _ = O.terrain_height(wt, 0.3, 0.4)
    assert O.ground_under(wt, 0.3, 0.4) == pytest.approx(h)
    assert O.ground_under(wt, 1.1, 0.0) == pytest.approx(0.3)   # the step box's top


def test_relative_height_cost_on_the_box():
    cfg = W.config_climb(K=1, H=2)
    w = O.World(cfg.robot)
    c = cfg.cost
    x = cfg.x0.astype(np.float64).copy()
    x[0], x[1], x[2] = 1.0, 0.0, 0.24 + c["z_ref"]
    x[22] = c["v_ref"]
    x[3:7] = [1, 0, 0, 0]
    cabs = dict(c, z_rel=0)
    # on the box at z_ref above its top: no height error relative to the ground, 0.24 absolute
    Lr = O.stage_costs(w, c, x[None], np.zeros((1, 12)), np.zeros(1))
    La = O.stage_costs(w, cabs, x[None], np.zeros((1, 12)), np.zeros(1))
    assert La[0] - Lr[0] == pytest.approx(c["w_z"] * 0.24 ** 2, rel=1e-12)
