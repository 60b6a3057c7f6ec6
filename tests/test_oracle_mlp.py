"""Pins of the FP64 proposal-network oracle: backprop gradient against central
finite differences (exact FP64 mode), GELU against its definition, BF16
rounding against known bit patterns, and an AdamW step against its formula on
a 1-parameter case."""
import math

import numpy as np

from oracle import mlp as M


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -2.5, 3.0e-5, 1 + 2 ** -9], np.float32)
    r = M.bf16(x)
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125 and r[3] == -2.5
    assert abs(r[4] - 3.0e-5) / 3.0e-5 < 2 ** -8
    assert r[5] == 1.0


def test_gelu_definition():
    z = np.linspace(-4, 4, 33)
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in z]))
    assert np.allclose(M.gelu(z), z * phi, atol=1e-15)
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-8)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = M.init_params(1).astype(np.float64)
    X = rng.normal(size=(5, 62))
    T = rng.normal(size=(5, 48))
    loss, g = M.loss_grad(p, X, T, mirror=False)
    idx = rng.choice(p.size, 60, replace=False)
    # include biases of every layer and corners of every weight block
    o = 0
    for no, ni in M.SIZES:
        idx = np.r_[idx, o, o + no * ni - 1, o + no * ni, o + no * ni + no - 1]
        o += no * ni + no
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_grad(pp, X, T, mirror=False)[0] - M.loss_grad(pm, X, T, mirror=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_mirror_close_to_exact():
    rng = np.random.default_rng(2)
    p = M.init_params(3)
    X = rng.normal(size=(16, 62))
    Y0, _ = M.forward(p, X, mirror=False)
    Y1, _ = M.forward(p, X, mirror=True)
    assert np.max(np.abs(Y1 - Y0)) <= 0.05 * np.max(np.abs(Y0))


def test_adamw_step_formula():
    p, m1, m2 = M.adamw(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, 0.1, 0.01)
    # first step: m_hat = g, v_hat = g^2 -> update = lr (sign(g) + wd p)
    assert np.allclose(p, 1.0 - 0.1 * (0.5 / (0.5 + 1e-8) + 0.01 * 1.0))
