"""Multi-instance benchmark (the persistent launch of many controllers).

The 16-instance mix of the multi-instance workload: heightfield terrain with the
0.3 m step box, K in {256 ... 4096}, H in {50, 100, 150} chosen by seed 2.  Each
block shape of the persistent kernel is timed over `steps` batch steps (CUDA
events on the batch's stream), then the autotuner picks one.  Prints one JSON
line: per-shape ms per batch step, the autotuned shape, and rollout-steps/s.

    python -m paper_2409_10469_gb300.multi [--steps N] [--instances N] [--shape 128x3]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import _mppi
from . import workloads as W

SHAPES = [(64, 1), (64, 2), (64, 4), (64, 6), (128, 1), (128, 2), (128, 3), (256, 1)]


def run(instances: int = 16, steps: int = 10, seed: int = 2, shapes=None, autotune: bool = True) -> dict:
    import torch
    mix = W.multi_instance_mix(instances, seed=seed)
    cfg = W.config_terrain()
    ctls = []
    for i, (K, H) in enumerate(mix):
        c = _mppi.Controller(cfg.robot, cfg.cost, dict(cfg.mppi, K=K, H=H, inst=i))
        c.set_nominal(cfg.mu0)
        ctls.append(c)
    stream = torch.cuda.Stream()
    batch = _mppi.Batch(ctls, stream=stream.cuda_stream)
    x0s = torch.zeros((instances, 50), device="cuda")
    x0s[:, :37] = torch.tensor(cfg.x0, dtype=torch.float32)
    per_shape = {}
    step = 0
    for blk, bpsm in (shapes or SHAPES):
        try:
            batch.set_shape(blk, bpsm)
        except _mppi.MppiError:
            continue          # above this block size's occupancy limit
        batch.step(x0s, np.full(instances, step, np.uint32))
        step += 1
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            batch.step(x0s, np.full(instances, step, np.uint32))
            step += 1
        e1.record(stream)
        torch.cuda.synchronize()
        per_shape["%dx%d" % (blk, bpsm)] = e0.elapsed_time(e1) / steps
    tuned = batch.autotune(x0s.cpu().numpy(), trials=3) if autotune else None
    best = min(per_shape.values())
    work = sum(K * H for K, H in mix)
    out = {"instances": instances, "mix_K_H": [list(m) for m in mix], "rollout_steps_per_batch_step": work,
           "ms_per_batch_step": per_shape, "autotune": list(tuned) if tuned is not None else None,
           "best_rollout_steps_per_s": work / (best * 1e-3)}
    batch.close()
    for c in ctls:
        c.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=16)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--shape", default=None, help="time one block shape only, e.g. 128x3 (no autotune)")
    a = ap.parse_args()
    from . import build as B
    B.build()           # the CUDA library (idempotent)
    shapes = [tuple(int(v) for v in a.shape.split("x"))] if a.shape else None
    print(json.dumps(run(a.instances, a.steps, a.seed, shapes=shapes, autotune=shapes is None)))


if __name__ == "__main__":
    main()
