"""Serving loop over the C ABI's continuous-batching runtime (mppi_server_*).

Simulated robots issue control-step requests at Poisson times; the loop
submits each request at its arrival time (or as soon as the robot's previous
request has completed), keeps calling the runtime's tick, and records every
request's latency from its arrival to its observed completion.  All GPU work
(sampling, rollouts, updates of every admitted request) runs in the library's
persistent multi-instance kernel; this module only schedules host calls.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import _mppi
from . import workloads as W


def build_robots(n_robots, seed, K_range=(512, 8192), H_range=(50, 150)):
    """Controllers of the serving workload (per-robot task, K, H); each robot has
    its own Philox stream (instance id = robot index)."""
    specs = W.serving_robots(n_robots, seed, K_range, H_range)
    ctls, x0s = [], []
    for r, (task, K, H) in enumerate(specs):
        cfg = W.task_config(task, K, H)
        m = dict(cfg.mppi, inst=r)
        c = _mppi.Controller(cfg.robot, cfg.cost, m)
        c.set_nominal(cfg.mu0)
        ctls.append(c)
        x0s.append(cfg.x0.astype(np.float32))
    return specs, ctls, x0s


def run(n_robots=64, rate_hz=50.0, duration=1.0, seed=4, budget_bytes=512 << 20,
        K_range=(512, 8192), H_range=(50, 150), warmup=0.1, capacity=False):
    """Serve Poisson arrivals for `duration` s; returns a metrics dict."""
    specs, ctls, x0s = build_robots(n_robots, seed, K_range, H_range)
    server = _mppi.Server(budget_bytes, n_robots, max(K for _, K, _ in specs))
    rids = [server.add_robot(c) for c in ctls]
    arrivals = W.serving_arrivals(n_robots, rate_hz, duration + warmup, seed)
    pending = collections.deque(arrivals)
    waiting = {r: collections.deque() for r in range(n_robots)}  # arrived, not yet submitted
    inflight = {}                                                # robot -> arrival time
    steps = np.zeros(n_robots, np.int64)
    lat, done_rs = [], 0.0
    t0 = time.perf_counter()
    while pending or any(waiting.values()) or inflight:
        now = time.perf_counter() - t0
        while pending and pending[0][0] <= now:
            t_arr, r = pending.popleft()
            waiting[r].append(t_arr)
        for r in range(n_robots):
            if waiting[r] and r not in inflight:
                t_arr = waiting[r].popleft()
                server.submit(rids[r], x0s[r], int(steps[r]))
                steps[r] += 1
                inflight[r] = t_arr
        server.tick()
        for r in list(inflight):
            res = server.poll(rids[r])
            if res is not None:
                t_arr = inflight.pop(r)
                t_done = time.perf_counter() - t0
                if t_arr >= warmup:
                    lat.append(t_done - t_arr)
                    _, K, H = specs[r]
                    done_rs += K * H
        if not pending and not any(waiting.values()) and not inflight:
            break
    elapsed = time.perf_counter() - t0 - warmup
    st = server.stats()
    lat = np.array(lat)
    offered = sum(K * H for t, r in arrivals if t >= warmup for (_, K, H) in [specs[r]])
    out = {
        "requests": int(len(lat)), "robots": n_robots, "rate_hz_per_robot": rate_hz,
        "duration_s": duration, "elapsed_s": elapsed,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                       "p99": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                       "max": float(lat.max() * 1e3) if len(lat) else None},
        "rollout_steps_per_s": done_rs / max(elapsed, 1e-9),
        "offered_rollout_steps_per_s": offered / duration,
        "launches": int(st["launches"]), "pool_peak_bytes": int(st["pool_peak"]),
        "budget_bytes": int(budget_bytes),
    }
    server.close()
    if capacity:
        out["capacity"] = batch_capacity(specs, ctls, x0s)
    for c in ctls:
        c.close()
    return out


def batch_capacity(specs, ctls, x0s, steps=10):
    """What the GPU sustains on this exact mix: every robot's solve in one
    persistent batch launch per step (autotuned block shape), CUDA events over
    `steps` steps -> rollout-steps/s; the serving rate is read against it."""
    import torch
    batch = _mppi.Batch(ctls)
    X = np.zeros((len(ctls), 50), np.float32)
    for i, x in enumerate(x0s):
        X[i, :len(x)] = x
    block, bpsm, _ = batch.autotune(X)
    batch.step(X, np.zeros(len(ctls), np.uint32))  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        batch.step(X, np.full(len(ctls), 1 + s, np.uint32))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    batch.close()
    work = sum(K * H for _, K, H in specs)
    return {"ms_per_batch_step": ms, "rollout_steps_per_s": work / (ms * 1e-3), "shape": [block, bpsm]}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="serving loop: Poisson requests of simulated robots")
    ap.add_argument("--robots", type=int, default=64)
    ap.add_argument("--rate", type=float, default=50.0, help="requests per second per robot")
    ap.add_argument("--duration", type=float, default=1.0, help="arrival window in seconds")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--budget-mb", type=int, default=512)
    ap.add_argument("--k-min", type=int, default=512)
    ap.add_argument("--k-max", type=int, default=8192)
    ap.add_argument("--capacity", action="store_true",
                    help="also time every robot's solve as one batch launch (the mix's GPU capacity)")
    a = ap.parse_args()
    from . import build as B
    B.build()
    print(json.dumps(run(n_robots=a.robots, rate_hz=a.rate, duration=a.duration, seed=a.seed,
                         budget_bytes=a.budget_mb << 20, K_range=(a.k_min, a.k_max), capacity=a.capacity)))


if __name__ == "__main__":
    main()
