"""The settings the paper states (tests/golden/paper_settings.json, each with
its citation) hold in the model spec: the oracle's knot representation, its
spline's degree, the workloads' control period and temperature, and the box
cost's norm.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_settings.json")))["values"]

CONFIGS = [W.config_stand, W.config_trot, W.config_trot_raibert, W.config_terrain, W.config_climb, W.config_push]


def test_knots_evenly_spaced_over_the_horizon():
    """Fig. 2 / Sec. IV-E: four knots per trajectory, evenly spaced: the
    parameter vector holds 4 x 12 joint targets and the spline passes through
    knot j at normalised time j / 3"""
    n = GOLDEN["knots_per_trajectory"]["value"]
    assert W.stand_mu().size == n * 12
    U = np.random.default_rng(0).uniform(-1, 1, n * 12).astype(np.float32)
    for j in range(n):
        assert np.allclose(O.spline_eval(U, j / (n - 1)), U.reshape(n, 12)[j].astype(np.float64), atol=1e-12)


def test_spline_degree_is_the_highest_through_the_knots():
    """Sec. III-B / IV-E: the cubic through four knots, the highest degree they
    fix: a cubic in tau is reproduced at every tau, a quartic is not"""
    deg = GOLDEN["interpolation_degree"]["value"]
    n = GOLDEN["knots_per_trajectory"]["value"]
    assert deg == n - 1
    tk = np.arange(n) / (n - 1)
    rng = np.random.default_rng(1)
    coef = rng.uniform(-0.5, 0.5, (12, deg + 1))
    f = lambda t, c: sum(c[:, p] * t ** p for p in range(c.shape[1]))
    U = np.stack([f(t, coef) for t in tk]).astype(np.float32)
    Ud = U.astype(np.float64)
    # the interpolant of the FP32 knots, checked against the cubic through them
    cub = np.stack([np.polyfit(tk, Ud[:, i], deg)[::-1] for i in range(12)])
    for tau in np.linspace(0, 1, 11):
        assert np.allclose(O.spline_eval(U.reshape(-1), tau), f(tau, cub), atol=1e-12)
    quart = np.concatenate([coef, np.full((12, 1), 0.7)], axis=1)
    Uq = np.stack([f(t, quart) for t in tk]).astype(np.float32)
    assert not np.allclose(O.spline_eval(Uq.reshape(-1), 0.5), f(0.5, quart), atol=1e-3)


@pytest.mark.parametrize("make", CONFIGS, ids=lambda f: f.__name__)
def test_control_rate_and_temperature(make):
    """Sec. IV-A / IV-E: the policy runs at 100 Hz (control period = ctrl_steps
    dt steps) with lambda = 0.1"""
    m = make().mppi
    assert m["ctrl_steps"] * m["dt"] == pytest.approx(1.0 / GOLDEN["policy_rate_hz"]["value"], abs=1e-12)
    assert m["lam"] == GOLDEN["temperature_lambda"]["value"]


def test_box_cost_is_l1():
    """Sec. IV-C: L_box = Q_box || x_goal - x_box ||_1 (xy): moving the box by
    (a, b) from its goal adds Q_box (|a| + |b|) to the stage cost"""
    assert GOLDEN["box_cost_norm"]["value"] == "l1"
    cfg = W.config_push()
    world = O.World(cfg.robot)
    gx, gy = cfg.cost["box_goal_xy"]
    X = np.tile(cfg.x0.astype(np.float64), (3, 1))
    X[:, 37], X[:, 38] = gx, gy
    X[1, 37:39] += (0.3, -0.2)
    X[2, 37:39] += (-0.1, 0.45)
    L = O.stage_costs(world, cfg.cost, X)
    q = cfg.cost["w_box"]
    assert L[1] - L[0] == pytest.approx(q * 0.5, rel=1e-12)
    assert L[2] - L[0] == pytest.approx(q * 0.55, rel=1e-12)
