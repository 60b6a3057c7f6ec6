"""Pins of the oracle's sampling step: Philox4x32-10 (Salmon et al., SC'11), the
project's FP32 ln / sincos against libm, Box-Muller normals against N(0, 1),
and the knot perturbation (Alg. 1 sampling step, Sec. II-B of arXiv 2409.10469)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import workloads as W


def ulp32(x):
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 2.0 ** (e - 23)


def test_lnf_exhaustive_on_sampling_domain():
    """All 2^24 uniforms u1 = n 2^-24, n = 1 .. 2^24: |lnf - ln| <= 2 ulp."""
    n = np.arange(1, 2 ** 24 + 1, dtype=np.float64)
    u = (n * 2.0 ** -24).astype(np.float32)
    y = O.lnf(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    err = np.abs(y - ref)
    nz = ref != 0
    assert np.all(err[nz] <= 2 * ulp32(ref[nz]))
    assert y[-1] == 0.0  # ln 1


def test_lnf_random_normal_floats():
    rng = np.random.default_rng(0)
    bits = rng.integers(0x00800000, 0x7f800000, 2_000_000, dtype=np.uint32)
    x = bits.view(np.float32)
    y = O.lnf(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    nz = np.abs(ref) > 1e-30
    assert np.all(np.abs(y - ref)[nz] <= 2 * ulp32(ref[nz]))


def test_sincos_exhaustive():
    """All 2^24 angles 2 pi n / 2^24: |cos - libm| and |sin - libm| <= 2 ulp of
    the result (exact zeros at the quarter turns)."""
    n = np.arange(2 ** 24, dtype=np.uint32)
    c, s = O.sincos_u24(n)
    th = 2 * np.pi * n.astype(np.float64) / 2 ** 24
    for got, ref in ((c, np.cos(th)), (s, np.sin(th))):
        got = got.astype(np.float64)
        err = np.abs(got - ref)
        big = np.abs(ref) > 1e-6
        assert np.all(err[big] <= 2 * ulp32(ref[big]))
        assert np.all(err[~big] <= 2 ** -24 * 1e-6 * 4 + 2e-13)
    assert c[0] == 1.0 and s[0] == 0.0
    q = 2 ** 22
    assert (c[q], s[q]) == (-0.0, 1.0) or (c[q] == 0 and s[q] == 1.0)
    assert c[2 * q] == -1.0 and s[2 * q] == 0 and c[3 * q] == 0 and s[3 * q] == -1.0


def test_philox_outputs_uniform_and_distinct():
    """Philox4x32-10 over consecutive counters: distinct words, uniform bytes
    (chi-square), balanced bits, and every input bit changes about half of the
    output bits (avalanche)."""
    outs = np.array([O.philox([i, 7, 3, 1], [0xDEADBEEF, 0x12345678]) for i in range(20000)])
    # 128-bit blocks are all distinct (32-bit words may collide: birthday bound)
    assert len(np.unique(outs, axis=0)) == outs.shape[0]
    by = outs.view(np.uint8).ravel()
    cnt = np.bincount(by, minlength=256)
    exp = by.size / 256
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 350  # 255 dof: mean 255, sd 22.6
    bits = np.unpackbits(outs.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.002
    base = O.philox([1, 2, 3, 4], [5, 6])
    flips = []
    for w in range(4):
        for b in range(32):
            c = [1, 2, 3, 4]
            c[w] ^= 1 << b
            d = O.philox(c, [5, 6]) ^ base
            flips.append(np.unpackbits(d.view(np.uint8)).sum())
    assert 56 < np.mean(flips) < 72


def test_philox_round_function_mulhilo():
    """One Philox round is a bijection built from 32x32->64 multiplies; check the
    key schedule effect: a key differing in one bit gives uncorrelated output."""
    a = O.philox([0, 0, 0, 0], [0, 0])
    b = O.philox([0, 0, 0, 0], [1, 0])
    assert np.unpackbits((a ^ b).view(np.uint8)).sum() > 40


def test_box_muller_normals_distribution():
    from scipy import stats
    eps = O.noise(0, 0, 0, np.arange(40000)).ravel().astype(np.float64)
    assert abs(eps.mean()) < 0.005
    assert abs(eps.var() - 1) < 0.01
    assert abs(stats.skew(eps)) < 0.02
    assert abs(stats.kurtosis(eps)) < 0.04
    assert stats.kstest(eps, "norm").pvalue > 1e-3
    # pairs are independent: correlation of the cos and sin halves ~ 0
    e = O.noise(0, 0, 0, np.arange(20000))
    assert abs(np.corrcoef(e[:, 0], e[:, 1])[0, 1]) < 0.03


def test_noise_streams_differ_by_step_instance_sample():
    a = O.noise(5, 0, 0, [3])
    assert not np.array_equal(a, O.noise(5, 1, 0, [3]))
    assert not np.array_equal(a, O.noise(5, 0, 1, [3]))
    assert not np.array_equal(a, O.noise(5, 0, 0, [4]))
    assert not np.array_equal(a, O.noise(6, 0, 0, [3]))
    assert np.array_equal(a, O.noise(5, 0, 0, [3]))


def test_sample_nominal_clamp_and_scale():
    m = W.mppi(512, 50, 0.01, 0.2, 8, seed=9)
    mu = W.stand_mu()
    U = O.sample(m, mu, step=3)
    assert np.array_equal(U[0], np.clip(mu, np.tile(W.Q_LO, 16), np.tile(W.Q_HI, 16)))
    lo = np.tile(np.array(W.Q_LO, np.float32), 16)
    hi = np.tile(np.array(W.Q_HI, np.float32), 16)
    assert np.all(U >= lo) and np.all(U <= hi)
    # unclamped entries are mu + sigma * eps exactly (fmaf) with eps the noise
    eps = O.noise(9, 3, 0, np.arange(1, 512))
    ref = np.clip((mu[None, :].astype(np.float64) + 0.2 * eps.astype(np.float64)), lo, hi)
    assert np.max(np.abs(U[1:] - ref)) < 1e-6
    z = ((U[1:] - mu) / 0.2)[(U[1:] > lo) & (U[1:] < hi)]
    assert abs(z.std() - 1) < 0.05


def test_sample_proposal_half():
    m = W.mppi(64, 50, 0.01, 0.2, 8, seed=1, n_prop=32)
    mu = W.stand_mu()
    mp = mu + 0.05
    U = O.sample(m, mu, 0, mu_prop=mp)
    assert np.array_equal(U[0], mu)
    assert np.array_equal(U[32], np.clip(mp, np.tile(W.Q_LO, 16), np.tile(W.Q_HI, 16)))
    assert abs(np.mean(U[33:] - mp)) < 0.02 and abs(np.mean(U[1:32] - mu)) < 0.02
