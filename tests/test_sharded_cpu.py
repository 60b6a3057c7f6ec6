"""The K-sharded control step's host protocol (paper_2409_10469_gb300.sharded)
on CPU: sample ranges that tile 0..K-1, and the all-reduce(min) + all-reduce(sum)
combination run over 2 and 4 gloo ranks, each rank's partial sums taken from
the FP64 oracle's rollouts of its own samples; every rank must end with the same
mean, equal to the oracle's Eq. 1 / Eq. 2 over all K samples (Alg. 1's samples
are independent until Eq. 1, whose weights factor through any shard minimum)."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2409_10469_gb300 import sharded as SH  # noqa: E402


@pytest.mark.parametrize("K", [1, 7, 64, 1000, 4096])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_ranges_tile_the_samples(K, world):
    seen = []
    for r in range(world):
        k0, n = SH.shard_range(K, r, world)
        seen.extend(range(k0, k0 + n))
        assert n in (K // world, K // world + 1)
    assert seen == list(range(K))


def partial_of(L, U, lam):
    """(m, Z, S): a shard's sums around its own finite-cost minimum, FP64"""
    L = np.asarray(L, np.float64)
    fin = np.isfinite(L)
    if not fin.any():
        return SH.empty_partial()
    m = L[fin].min()
    w = np.where(fin, np.exp(-(np.where(fin, L, m) - m) / lam), 0.0)
    return np.concatenate([[m, w.sum()], w @ np.asarray(U, np.float64)])


def test_combine_equals_the_unsharded_weights():
    """in one process (a list stands in for the ranks): the factor scaling
    reproduces exp(-(L - L_min)/lambda) over all samples, with one shard whose
    costs are all non-finite"""
    rng = np.random.default_rng(0)
    K, lam = 100, 0.1
    L = 50 + 30 * rng.random(K)
    L[40:55] = np.inf
    U = rng.normal(size=(K, 48))
    shards = [(0, 40), (40, 15), (55, 45)]
    parts = [partial_of(L[k0:k0 + n], U[k0:k0 + n], lam) for k0, n in shards]
    for p in parts:
        sums = SH.combine(p, lam, lambda v: min(q[0] for q in parts),
                          lambda a: sum(math.exp(-(q[0] - min(r[0] for r in parts)) / lam) * q[1:]
                                        if math.isfinite(q[0]) else 0 * q[1:] for q in parts))
        fin = np.isfinite(L)
        w = np.where(fin, np.exp(-(np.where(fin, L, 0) - L[fin].min()) / lam), 0.0)
        assert sums[0] == pytest.approx(w.sum(), rel=1e-13)
        assert np.allclose(sums[1:], w @ U, rtol=1e-12, atol=1e-12)


class OracleShardEngine:
    """a rank's stand-in for a controller handle: its samples' knots are the
    oracle's Philox samples and their costs the oracle's rollouts (FP32, as the
    kernels return them); the partial sums as mppi_step_partial defines them"""

    def __init__(self, cfg, m):
        import oracle as O
        self.O, self.cfg, self.m = O, cfg, m
        self.K, self.lam = m["K"], m["lam"]
        self.mu = cfg.mu0.astype(np.float32)
        self.world = O.World(cfg.robot)

    def samples(self, step, k0, n, x0):
        U = self.O.sample(self.m, self.mu, step)[k0:k0 + n]
        t0 = step * self.m["ctrl_steps"] * self.m["dt"]
        L = self.O.rollouts(self.world, self.cfg.cost, self.m, t0, np.asarray(x0, np.float64), U)
        return U, L.astype(np.float32)

    def step_partial(self, x0, step, k0, n):
        U, L = self.samples(step, k0, n, x0)
        return partial_of(L, U, self.lam)

    def step_finalize(self, sums, u0_out=None, mu_out=None, check=False):
        self.mu_new = (np.asarray(sums[1:]) / sums[0]).astype(np.float32)
        return 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2409_10469_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = W.config_stand(K=60, H=12)
    eng = OracleShardEngine(cfg, dict(cfg.mppi))
    x0 = cfg.x0.astype(np.float32)
    SH.sharded_step(eng, x0, 3, rank, world, SH.torch_reducers())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, eng.mu_new))


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_step_over_gloo_ranks_equals_the_oracle_update(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank holds the same mean ...
    for r in range(1, world):
        assert np.array_equal(out[r], out[0])
    # ... the oracle's Eq. 1 / Eq. 2 over all K samples of the step
    import oracle as O
    from paper_2409_10469_gb300 import workloads as W
    cfg = W.config_stand(K=60, H=12)
    eng = OracleShardEngine(cfg, dict(cfg.mppi))
    U, L = eng.samples(3, 0, 60, cfg.x0.astype(np.float32))
    _, mu_o, _ = O.update(L, U, cfg.mppi["lam"])
    assert np.max(np.abs(out[0] - mu_o) / np.maximum(np.abs(mu_o), 1.0)) <= 1e-6
