"""The operation-counting build of the oracle (real = a counting scalar): it
runs the same arithmetic as the FP64 oracle, and its count of the plain
formulation's floating-point work bounds the structured count the roofline
uses (flops.py) from above."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10469_gb300 import flops as F, workloads as W


def _trot():
    cfg = W.config_trot(K=4096, H=100)
    return cfg, cfg.mppi


def test_counting_build_is_the_fp64_oracle():
    cfg, m = _trot()
    rng = np.random.default_rng(5)
    x0 = cfg.x0.astype(np.float64)
    X = np.repeat(x0[None], 4, 0)
    X[:, 7:19] += rng.uniform(-0.2, 0.2, (4, 12))
    X[:, 25:37] += rng.uniform(-1, 1, (4, 12))
    Ut = np.repeat(cfg.mu0[None, :12].astype(np.float64), 4, 0)
    h = m["dt"] / m["n_sub"]
    ref = O.dt_steps(O.World(cfg.robot), X, Ut, m["n_sub"], h, nthreads=1)
    with O.use_count():
        got = O.dt_steps(O.World(cfg.robot), X, Ut, m["n_sub"], h, nthreads=1)
    assert np.array_equal(got, ref)


def test_counted_plain_flops_per_substep():
    cfg, m = _trot()
    with O.use_count() as cnt:
        world = O.World(cfg.robot)
        x0 = cfg.x0.astype(np.float64)
        Ut = cfg.mu0[None, :12].astype(np.float64)
        cnt.opcounts()
        O.dt_steps(world, x0[None], Ut, m["n_sub"], m["dt"] / m["n_sub"], nthreads=1)
        c = cnt.opcounts()
    per_sub = (c["add"] + c["mul"] + c["div"] + c["sqrt"]) / m["n_sub"]
    # the recorded figure (flops.py) is this count, and it bounds the structured
    # formulation the kernel implements from above
    assert per_sub == pytest.approx(F.ORACLE_PLAIN_SUBSTEP, rel=0.02)
    assert F.SUBSTEP < per_sub
    assert c["trans"] > 0 and c["sqrt"] > 0
