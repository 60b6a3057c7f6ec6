"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own instance
id; the timing protocol (barrier, max over ranks) and the weak-scaling
throughput of paper_2409_10469_gb300.dist."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2409_10469_gb300 import dist as D
    r, w, lr = D.env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    t = 0.010 * (r + 1)                     # rank 1 is the slow one
    tmax = D.max_over_ranks(t)
    value = D.job_throughput(4096 * 100, w, tmax)
    # every rank's instance id differs (independent Philox streams)
    ids = [None] * w
    dist.all_gather_object(ids, r)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, tmax, value, ids))


def test_two_rank_timing_protocol():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, tmax, value, ids in out:
        assert tmax == pytest.approx(0.020)
        assert value == pytest.approx(2 * 4096 * 100 / 0.020)
        assert sorted(ids) == [0, 1]
