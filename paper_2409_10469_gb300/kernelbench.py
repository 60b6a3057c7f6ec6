"""Timing of the HBM-bound kernels on their own calls: the sampler (mppi_sample)
and the update (mppi_update) of a controller at K samples, for the knot
representations (48 parameters per sample) or direct targets (12 H), with the
L2 flushed between calls (a 256 MB write) and CUDA events on the current stream.
A spin kernel (about 100 us) runs ahead of the first event of each call, so the
host's time to enqueue the call's kernels overlaps it and the events bracket
device time only.

    python -m paper_2409_10469_gb300.kernelbench --K 16384 --H 100 --interp direct
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def run(K: int, H: int, interp: str = "direct", calls: int = 12, warmup: int = 3) -> dict:
    import torch

    from . import _mppi, build as B, flops as F, workloads as W
    B.build()
    cfg = W.config_trot(K=K, H=H)
    ctl = _mppi.Controller(cfg.robot, cfg.cost, dict(cfg.mppi, interp=interp))
    D = ctl.D
    rng = np.random.default_rng(0)
    U = torch.tensor(rng.normal(0.5, 0.3, (K, D)).astype(np.float32)).cuda()
    L = torch.tensor((100 + 50 * rng.random(K)).astype(np.float32)).cuda()
    U2 = torch.empty((K, D), device="cuda")
    flush = torch.empty(64 << 20, device="cuda")
    t_upd, t_smp = [], []
    for s in range(warmup + calls):
        # the update's kernels alone: its outputs stay in the handle (no copies)
        for fn, out in ((lambda: ctl.update(L, U, n=K), t_upd),
                        (lambda: ctl.sample(s, out=U2), t_smp)):
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda._sleep(200000)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            if s >= warmup:
                out.append(e0.elapsed_time(e1))
    ctl.close()
    tu, ts = float(np.mean(t_upd)), float(np.mean(t_smp))
    bu, bs = F.update_bytes(K, D), F.sample_bytes(K, D)
    return {"K": K, "H": H, "interp": interp, "params_per_sample": D,
            "update": {"us": tu * 1e3, "bytes": bu, "TB_per_s": bu / (tu * 1e-3) / 1e12},
            "sample": {"us": ts * 1e3, "bytes": bs, "TB_per_s": bs / (ts * 1e-3) / 1e12}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=16384)
    ap.add_argument("--H", type=int, default=100)
    ap.add_argument("--interp", default="direct")
    ap.add_argument("--calls", type=int, default=12)
    a = ap.parse_args()
    print(json.dumps(run(a.K, a.H, a.interp, a.calls)))


if __name__ == "__main__":
    main()
