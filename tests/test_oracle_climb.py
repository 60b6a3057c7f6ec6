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


@pytest.mark.parametrize("vx", [0.0, 0.5, 1.2, -0.3, 5.0])
@pytest.mark.parametrize("t", [0.0, 0.06, 0.13, 0.31, 0.44])
def test_raibert_reference_closed_form(vx, t):
    c = W.cost("trot_raibert")
    c1 = dict(c, gait=1)
    P, k, Lg, vr = c["gait_period"], c["raibert_k"], c["raibert_len"], c["v_ref"]
    dth = min(0.4, max(-0.4, -(P / 4 * vx + k * (vx - vr)) / Lg))
    u2 = O.gait_ref_x(c, t, state_with_vx(vx))
    u1 = O.gait_ref(c1, t)
    phase0 = [0, 1, 1, 0]
    for leg in range(4):
        s = math.sin(2 * math.pi * t / P + math.pi * phase0[leg])
        sw = max(0.0, s)
        # abduction and knee as in the open-loop trot; hip moved by sw * dth
        assert u2[3 * leg] == u1[3 * leg] and abs(u2[3 * leg + 2] - u1[3 * leg + 2]) < 1e-15
        assert abs(u2[3 * leg + 1] - (u1[3 * leg + 1] + sw * dth)) < 1e-12
        if s <= 0:
            assert u2[3 * leg + 1] == u1[3 * leg + 1]      # stance legs carry no feedback


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
