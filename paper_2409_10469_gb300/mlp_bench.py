"""Benchmark of the proposal network's tensor-core path.

Times (CUDA events) the BF16 tcgen05 GEMM D = A B^T of the network's shapes at
several row counts, and one forward / one training step of the 62 -> 256 ->
256 -> 256 -> 48 network at several batch sizes.  Prints one JSON line: per
shape ms, TFLOP/s (2 M N K per GEMM) and the fraction of the measured dense
BF16 peak (MEASURED_PEAKS.json, else 1.9 PFLOP/s).

    python -m paper_2409_10469_gb300.mlp_bench
    python -m paper_2409_10469_gb300.mlp_bench --train 4096 --steps 3   # training steps only
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import _mppi
from . import workloads as W

GEMMS = [(512, 256, 256), (4096, 256, 256), (16384, 256, 256), (65536, 256, 256), (65536, 256, 64),
         (65536, 64, 256)]
BATCHES = [8, 64, 512, 4096]


def _peak_tflops():
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops"
    return 1900.0, "fallback 1.9 PFLOP/s"


def _time(fn, reps=20):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run() -> dict:
    import torch
    peak, src = _peak_tflops()
    g = torch.Generator(device="cuda").manual_seed(0)
    out = {"gemm": {}, "mlp": {}, "peak_tflops": peak, "peak_source": src}
    for M, N, K in GEMMS:
        A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
        D = torch.empty((M, N), device="cuda")
        Ab, Bb = A.view(torch.int16), B.view(torch.int16)
        ms = _time(lambda: _mppi.tc_gemm_bf16(Ab, Bb, M, N, K, D))
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out["gemm"]["%dx%dx%d" % (M, N, K)] = {"ms": ms, "tflops": tf, "frac": tf / peak}
    for Bn in BATCHES:
        net = _mppi.MLP(Bn)
        net.set_params(W.mlp_init(0))
        X = torch.randn((Bn, 62), device="cuda", generator=g)
        T = torch.randn((Bn, 48), device="cuda", generator=g)
        Y = torch.empty((Bn, 48), device="cuda")
        fwd = _time(lambda: net.forward(X, out=Y))
        trn = _time(lambda: net.train_step(X, T, lr=1e-4))
        out["mlp"]["batch%d" % Bn] = {"forward_ms": fwd, "train_step_ms": trn}
        net.close()
    return out


def train_steps(batch: int, steps: int) -> dict:
    """`steps` training steps of the network at one batch size (the launch
    sequence a profiler captures); returns the last loss"""
    import torch
    g = torch.Generator(device="cuda").manual_seed(0)
    net = _mppi.MLP(batch)
    net.set_params(W.mlp_init(0))
    X = torch.randn((batch, 62), device="cuda", generator=g)
    T = torch.randn((batch, 48), device="cuda", generator=g)
    loss = None
    for _ in range(steps):
        loss = net.train_step(X, T, lr=1e-4)
    torch.cuda.synchronize()
    net.close()
    return {"batch": batch, "steps": steps, "loss": float(loss)}


def main():
    import argparse
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--train", type=int, default=0, help="only run training steps at this batch size")
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args()
    from . import build as B
    B.build()
    if args.train:
        print(json.dumps(train_steps(args.train, args.steps)))
    else:
        print(json.dumps(run()))


if __name__ == "__main__":
    main()
