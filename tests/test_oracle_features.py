"""Pins of the oracle's 62 proposal-network input features (oracle/features.py)
against values fixed by hand on constructed states: the learned proposal's
inputs (pattern 4; the paper's Sec. V-B names better sampling distributions as
future work) are a model-spec choice, so each pin is a state whose features are
known without evaluating the definition -- a level robot at rest, a pitched
trunk (the world's vertical seen from the body is the rotation's third row), a
yawed box (its heading), known robot / box / goal positions, and the gait
phase at known fractions of the period."""
import math

import numpy as np
import pytest

from oracle import features as F
from paper_2409_10469_gb300 import workloads as W

STAND = np.array(W.STAND, np.float64)


def push_cost(goal=(0.0, 0.0), box_goal=(0.0, 0.0), gait=0, period=0.5):
    c = W.cost("stand")
    return dict(c, goal_xy=goal, box_goal_xy=box_goal, gait=gait, gait_period=period)


def test_level_robot_at_rest_at_the_origin():
    x = W.stand_state(z=0.3)
    f = F.features(x, push_cost(goal=(1.5, -0.5)), ctrl_steps=2, dt=0.005, step=0)
    assert f[0] == 0.3
    assert np.array_equal(f[1:5], [1, 0, 0, 0])
    assert np.array_equal(f[5:17], np.tile(STAND, 4))
    assert np.all(f[17:35] == 0)                       # trunk and joint velocities
    assert np.all(f[35:50] == 0)                       # no box
    assert np.array_equal(f[50:52], [1.5, -0.5])       # goal offset from the trunk
    assert (f[52], f[53]) == (0.0, 1.0)                # stand: no gait phase
    assert np.array_equal(f[54:57], [0, 0, 1])         # the world's vertical in the body frame
    assert np.all(f[57:61] == 0)
    assert f[61] == 1.0


def test_quaternion_sign_is_canonical():
    x = W.stand_state()
    x[3:7] = [0.9, 0.1, -0.3, 0.2]
    x[3:7] /= np.linalg.norm(x[3:7])
    y = x.copy()
    y[3:7] = -x[3:7]
    c = push_cost()
    fx, fy = F.features(x, c, 2, 0.005, 0), F.features(y, c, 2, 0.005, 0)
    assert np.array_equal(fx, fy)
    assert fx[1] > 0


@pytest.mark.parametrize("theta", [0.3, -0.7, 1.2])
def test_pitched_trunk_sees_gravity_tilted(theta):
    """pitch theta about the body y axis: quaternion (cos theta/2, 0, sin theta/2, 0);
    the world's e_z in body coordinates is (-sin theta, 0, cos theta)"""
    x = W.stand_state()
    x[3:7] = [math.cos(theta / 2), 0, math.sin(theta / 2), 0]
    f = F.features(x, push_cost(), 2, 0.005, 0)
    assert f[54:57] == pytest.approx([-math.sin(theta), 0.0, math.cos(theta)], abs=1e-15)


@pytest.mark.parametrize("phi", [0.4, -1.1])
def test_rolled_trunk_sees_gravity_tilted(phi):
    """roll phi about the body x axis: the world's e_z in body coordinates is
    (0, sin phi, cos phi)"""
    x = W.stand_state()
    x[3:7] = [math.cos(phi / 2), math.sin(phi / 2), 0, 0]
    f = F.features(x, push_cost(), 2, 0.005, 0)
    assert f[54:57] == pytest.approx([0.0, math.sin(phi), math.cos(phi)], abs=1e-15)


@pytest.mark.parametrize("psi", [0.0, 0.5, 2.0, -2.5])
def test_yawed_box_heading(psi):
    """a box yawed by psi about the vertical: quaternion (cos psi/2, 0, 0, sin psi/2);
    its heading features are (cos psi, sin psi)"""
    x = W.stand_state(box_xy=(0.6, 0.0))
    x[40:44] = [math.cos(psi / 2), 0, 0, math.sin(psi / 2)]
    f = F.features(x, push_cost(), 2, 0.005, 0)
    assert f[57:59] == pytest.approx([math.cos(psi), math.sin(psi)], abs=1e-15)


def test_known_robot_box_and_goal_positions():
    x = W.stand_state(z=0.31, box_xy=(1.5, 2.5))
    x[0:2] = (1.0, 2.0)
    x[39] = 0.2
    x[44:50] = [0.1, -0.2, 0.3, 0.4, -0.5, 0.6]      # box angular and linear velocity
    x[25:37] = np.arange(12)                          # joint rates
    f = F.features(x, push_cost(goal=(0.5, 0.0), box_goal=(3.0, 4.0)), 2, 0.005, 0)
    assert np.array_equal(f[35:37], [0.5, 0.5])       # box relative to the trunk
    assert f[37] == 0.2                               # box height
    assert np.array_equal(f[38:42], [1, 0, 0, 0])
    assert np.array_equal(f[42:48], [0.1, -0.2, 0.3, 0.4, -0.5, 0.6])
    assert np.array_equal(f[48:50], [1.5, 1.5])       # box goal relative to the box
    assert np.array_equal(f[50:52], [-0.5, -2.0])     # robot goal relative to the trunk
    assert f[59] == pytest.approx(1.5 * math.sqrt(2), abs=1e-15)
    assert f[60] == pytest.approx(0.5 * math.sqrt(2), abs=1e-15)
    assert f[23:35] == pytest.approx(0.1 * np.arange(12), abs=1e-15)


@pytest.mark.parametrize("step,expect", [(0, (0.0, 1.0)), (25, (1.0, 0.0)), (50, (0.0, -1.0)),
                                          (75, (-1.0, 0.0)), (100, (0.0, 1.0)), (125, (1.0, 0.0))])
def test_gait_phase_at_known_fractions_of_the_period(step, expect):
    """trot gait, period 0.5 s, control period 5 ms: step 25 is a quarter period
    (phase pi/2), step 50 half of it, step 100 a whole one (wrapped)"""
    x = W.stand_state()
    f = F.features(x, push_cost(gait=1), ctrl_steps=1, dt=0.005, step=step)
    assert (f[52], f[53]) == pytest.approx(expect, abs=1e-12)
