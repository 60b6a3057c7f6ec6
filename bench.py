"""Benchmark of one MPPI control step (arXiv 2409.10469, Alg. 1) on GB300.

Workload: trot on a flat plane (dt 0.005 s, n_sub 8, sigma 0.3, lambda 0.1)
at K = 4096 samples, H = 100 steps.  A step is one full pass of the hot path:
Philox knot sampling (inside the rollout kernel) -> 4096 rollouts of the floating-base quadruped ->
softmax update, applied control and shift (mppi_step of the C ABI).

Metric: rollout-steps/s = K * H / step time (plus step latency p50 / p99).
`value` is device-timed with inputs resident in HBM (CUDA events around each
step on the controller's stream, L2 flushed between steps outside the timed
events); `e2e` times the same call through the C ABI with HOST buffers (x0
copied in from pinned memory, u0 read back) on the host clock.

`--impl reference` times the FP64 CPU oracle on the host cores on the same
workload and config (each step all K rollouts, or as many as keep the run
within about two minutes).  Under torchrun each
rank runs its own independent controller instance (weak scaling, no
collective: MPPI instances share nothing).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_BENCH, H_BENCH = 4096, 100
METRIC = "rollout-steps/s (MPPI step, K=4096, H=100)"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture) of
# one k_rollout launch on this workload, valid only for the kernel sources whose
# SHA-256 prefix is given; reported as null once those sources change.
ROLLOUT_TRAFFIC = {"bytes": 106240, "sources_sha256": "6d12a4c3579f2422"}
ROLLOUT_SOURCES = ("rollout.cu", "rollout.cuh", "common.cuh", "noise.cuh", "kernels.h", "precise.cuh")


def rollout_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in ROLLOUT_SOURCES:
        with open(os.path.join(ROOT, "paper_2409_10469_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    ok = h.hexdigest()[:16] == ROLLOUT_TRAFFIC["sources_sha256"]
    return ROLLOUT_TRAFFIC["bytes"] if ok else None


def bench_config(n_sub):
    """The workload both arms run (the GPU arm and --impl reference)."""
    return {"workload": "trot flat plane K=4096 H=100 dt=0.005 n_sub=%d" % n_sub,
            "K": K_BENCH, "H": H_BENCH, "n_sub": n_sub,
            "l2": "GPU arm: L2 flushed between steps; reference arm: host, no GPU",
            "parallelism": "independent instance per GPU"}


def dist_env():
    from paper_2409_10469_gb300 import dist as D
    return D.env()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every `period_ms` by one
    `nvidia-smi -lms` process started before the warm-up; the summary keeps the
    samples that fall inside the timed region (marked by `window()`)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.idx = gpu_index
        self.period_ms = period_ms
        self.rows = []          # (host time, fields)
        self.t0 = self.t1 = None
        self._p = None
        self._t = None

    def _read(self):
        for line in self._p.stdout:
            f = [x.strip() for x in line.strip().split(",")]
            if len(f) >= 9:
                self.rows.append((time.perf_counter(), f))

    def start(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                        "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._p = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        return self

    def stop(self):
        if self._p is not None:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
            self._t.join(timeout=5)
            self._p = None

    class _Window:
        def __init__(self, s):
            self.s = s

        def __enter__(self):
            self.s.t0 = time.perf_counter()

        def __exit__(self, *a):
            self.s.t1 = time.perf_counter()

    def window(self):
        return ClockSampler._Window(self)

    def summary(self):
        rows = [f for t, f in self.rows
                if self.t0 is not None and self.t1 is not None and self.t0 - 0.06 <= t <= self.t1 + 0.06]
        where = "timed region"
        if not rows and self.rows:   # region shorter than the sampling period: the nearest samples
            mid = 0.5 * (self.t0 + self.t1) if self.t0 is not None and self.t1 is not None else 0.0
            rows = [f for t, f in sorted(self.rows, key=lambda r: abs(r[0] - mid))[:2]]
            where = "nearest to the timed region"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows), "sampled": where, "period_ms": self.period_ms}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def _oracle_rate(O, cfg, seconds, cores):
    world = O.World(cfg.robot)
    m = dict(cfg.mppi)
    U = O.sample(dict(m, K=256), cfg.mu0, 0)
    x0 = cfg.x0.astype(np.float64)
    n_roll, t_start = 0, time.perf_counter()
    while True:
        O.rollouts(world, cfg.cost, m, 0.0, x0, U, nthreads=cores)
        n_roll += U.shape[0]
        el = time.perf_counter() - t_start
        if el >= seconds:
            break
    return n_roll * m["H"] / el, n_roll, el


def cpu_baseline(cfg, seconds=12.0):
    """The oracle as it stands, on all host cores, over a bounded sample of the
    workload's rollouts (whole batches of 256 until the time is used): the FP64
    build (the reported value) for 2/3 of `seconds`, the FP32 build of the same
    source for the rest."""
    import oracle as O
    cores = os.cpu_count() or 1
    m = cfg.mppi
    rate, n_roll, el = _oracle_rate(O, cfg, seconds * 2 / 3, cores)
    with O.use_float():
        rate32, n32, el32 = _oracle_rate(O, cfg, seconds / 3, cores)
    return {"value": rate, "unit": "rollout-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d rollouts of the K=4096 H=100 trot workload (H=%d, n_sub=%d, FP64) in %.1f s"
                      % (n_roll, m["H"], m["n_sub"], el),
            "fp32_build": {"value": rate32, "unit": "rollout-steps/s",
                           "sample": "%d rollouts, same source compiled with real = float, in %.1f s"
                                     % (n32, el32)}}


def run_reference(args):
    """--impl reference: the FP64 oracle on host cores, same workload, metric and
    config.  A step rolls out as many of the K samples as keeps the whole run
    (warm-up included) within about two minutes -- all K when that fits -- and
    ms_per_step is the measured time of such a step."""
    rank, world_size, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_2409_10469_gb300 import workloads as W
    cfg = W.config_trot(K=K_BENCH, H=H_BENCH)
    world = O.World(cfg.robot)
    cores = os.cpu_count() or 1
    m = dict(cfg.mppi)
    x0 = cfg.x0.astype(np.float64)
    mu = cfg.mu0.copy()
    # rollouts per step: rate calibrated on 64 rollouts, ~2 minutes for the run
    t = time.perf_counter()
    O.rollouts(world, cfg.cost, m, 0.0, x0, O.sample(dict(m, K=64), mu, 0), nthreads=cores)
    per_rollout = (time.perf_counter() - t) / 64
    budget = 120.0 / max(1, args.steps + args.warmup)
    sample_K = int(max(16, min(K_BENCH, budget / per_rollout)))

    def one(step):
        U = O.sample(dict(m, K=sample_K), mu, step)
        t = time.perf_counter()
        L = O.rollouts(world, cfg.cost, m, 0.0, x0, U, nthreads=cores)
        O.update(L.astype(np.float32), U, m["lam"])
        return time.perf_counter() - t

    for s in range(args.warmup):
        one(s)
    times = [one(args.warmup + s) for s in range(args.steps)]
    per_step = float(np.mean(times))
    value = sample_K * H_BENCH / per_step
    sample = ("all %d rollouts of the step" % K_BENCH if sample_K == K_BENCH else
              "%d of the %d rollouts per step (the run bounded to ~2 minutes)" % (sample_K, K_BENCH))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rollout-steps/s",
            "n_gpus": world_size, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(m["n_sub"]),
            "rollouts_per_step": sample_K,
            "cpu_baseline": {"value": value, "unit": "rollout-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "rollout-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def hbm_line(nbytes, ms, peaks):
    """An HBM roofline entry for a byte-moving kernel: algorithmic bytes over its
    CUDA-event time against the measured copy bandwidth."""
    peak = (peaks or {}).get("hbm_gbs", 6800.0)
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_launch": nbytes, "ms": ms,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}


def component_ms(ctl, stream, flush, K, reps=16):
    """The noise kernel (mppi_sample) and the update kernel (mppi_update) timed on
    their own calls at the bench's K (the control step runs both inside its one
    kernel): CUDA events on the controller's stream, L2 flushed between calls"""
    import torch
    U = torch.empty((K, 48), dtype=torch.float32, device="cuda")
    L = torch.rand(K, dtype=torch.float32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    mu = torch.empty(48, dtype=torch.float32, device="cuda")
    out = {"k_sample": [], "k_update": []}
    for r in range(reps + 2):
        for name, call in (("k_sample", lambda: ctl.sample(50000 + r, out=U)),
                           ("k_update", lambda: ctl.update(L, U, n=K, mu_out=mu))):
            with torch.cuda.stream(stream):
                flush.fill_(float(r))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            stream.synchronize()
            if r >= 2:
                out[name].append(e0.elapsed_time(e1))
    return {k: float(np.mean(v)) for k, v in out.items()}


def full_occupancy_roofline(cfg_fn, F, flush, peak, n_sm, steps=30):
    """The same step at K = 2 x SMs x 32 (9728 on 152 SMs): CTAs of 128 threads,
    two per SM (the kernel's register budget allows two), so every scheduler
    runs two warps -- at the metric's K = 4096 only 512 warps exist for 608
    schedulers.  CUDA events around each step, L2 flushed between steps."""
    import torch
    from paper_2409_10469_gb300 import _mppi
    K = 2 * n_sm * 32
    cfg = cfg_fn(K=K, H=H_BENCH)
    st = torch.cuda.Stream()
    ctl = _mppi.Controller(cfg.robot, cfg.cost, cfg.mppi, stream=st.cuda_stream)
    ctl.set_nominal(cfg.mu0)
    x0 = torch.tensor(cfg.x0, dtype=torch.float32, device="cuda")
    u0 = torch.empty(12, dtype=torch.float32, device="cuda")
    for s in range(3):
        ctl.step(x0, s, u0_out=u0)
    ms = []
    for s in range(steps):
        with torch.cuda.stream(st):
            flush.fill_(float(s))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctl.step(x0, 3 + s, u0_out=u0)
        e1.record(st)
        st.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctl.close()
    t = float(np.mean(ms))
    ach = F.rollout_flops(K, H_BENCH, cfg.mppi["n_sub"]) / (t * 1e-3) / 1e12
    return {"K": K, "H": H_BENCH, "ms_per_step": t, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "note": "same kernel, two warps per scheduler (the metric's K = 4096 fills one)"}


def proposal_form(flush, steps=200, warmup=10):
    """The learned-proposal form beside the plain one: the same trot workload at
    K = 2048 with half the samples drawn around the network's mean (random-init
    weights of the network's architecture; timing does not depend on them).  One
    control step = the features of the current state, the network's forward
    (small-batch kernel), the proposal handed to the controller, and the control
    step (one kernel) -- all device-resident on one stream, enqueued by one call;
    timed too as the four separate calls.  CUDA events around each step, L2
    flushed between steps."""
    import torch
    from paper_2409_10469_gb300 import _mppi, workloads as W
    K = K_BENCH // 2
    cfg = W.config_trot(K=K, H=H_BENCH)
    m = dict(cfg.mppi, n_prop=K // 2)
    st = torch.cuda.Stream()
    ctl = _mppi.Controller(cfg.robot, cfg.cost, m, stream=st.cuda_stream)
    ctl.set_nominal(cfg.mu0)
    net = _mppi.MLP(1, stream=st.cuda_stream)
    net.set_params(W.mlp_init(0))
    x0 = torch.tensor(cfg.x0, dtype=torch.float32, device="cuda")
    feat = torch.empty((1, 62), dtype=torch.float32, device="cuda")
    mu_p = torch.empty((1, 48), dtype=torch.float32, device="cuda")
    u0 = torch.empty(12, dtype=torch.float32, device="cuda")

    def four(s):
        ctl.features(x0[None], s, out=feat)
        net.forward(feat, out=mu_p)
        ctl.set_proposal(mu_p[0])
        ctl.step(x0, s, u0_out=u0)

    def one(s):
        ctl.step_proposal(net, x0, s, u0_out=u0)

    def timed(fn):
        for s in range(warmup):
            fn(s)
        st.synchronize()
        ms = []
        for s in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(warmup + s)
            e1.record(st)
            st.synchronize()
            ms.append(e0.elapsed_time(e1))
        return np.array(ms)

    ms4 = timed(four)
    ms = timed(one)
    net.close()
    ctl.close()
    t = float(ms.mean())
    return {"K": K, "n_prop": K // 2, "H": H_BENCH, "ms_per_step": t,
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "rollout_steps_per_s": K * H_BENCH / (t * 1e-3),
            "four_calls_ms_per_step": float(ms4.mean()),
            "step": "mppi_step_proposal: features + network forward + proposal + control step in one call "
                    "on one stream (four_calls: the same as four separate calls)"}


def direct_form(flush, peaks, steps=60, warmup=5):
    """Direct targets (the paper's sampling ablation, Sec. IV-E): the same trot
    workload at K = 4096, H = 100 with 12 H = 1200 sampled parameters per
    sample instead of 48 knots.  The step is three stages (sampling, rollouts,
    and the update's three launches: L_min, the row-streaming sums, the
    combine), each timed by the library's CUDA events on the stream
    (mppi_set_timing); L2 flushed between steps.  The sampler writes and the
    update reads 19.7 MB per step, so these two are HBM stages."""
    import torch
    from paper_2409_10469_gb300 import _mppi, flops as F, workloads as W
    K, H = K_BENCH, H_BENCH
    Dp = 12 * H
    cfg = W.config_trot(K=K, H=H)
    st = torch.cuda.Stream()
    ctl = _mppi.Controller(cfg.robot, cfg.cost, dict(cfg.mppi, interp="direct"), stream=st.cuda_stream)
    ctl.set_nominal(np.tile(W.stand_mu()[:12], H).astype(np.float32))
    ctl.set_timing(True)
    x0 = torch.tensor(cfg.x0, dtype=torch.float32, device="cuda")
    u0 = torch.empty(12, dtype=torch.float32, device="cuda")
    for s in range(warmup):
        ctl.step(x0, s, u0_out=u0)
    st.synchronize()
    ms, parts = [], []
    for s in range(steps):
        with torch.cuda.stream(st):
            flush.fill_(float(s))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctl.step(x0, warmup + s, u0_out=u0)
        e1.record(st)
        st.synchronize()
        ms.append(e0.elapsed_time(e1))
        parts.append(ctl.timings())
    ctl.close()
    p = np.mean(np.array(parts), axis=0)
    t = float(np.mean(ms))
    return {"K": K, "H": H, "params_per_sample": Dp, "ms_per_step": t,
            "rollout_steps_per_s": K * H / (t * 1e-3),
            "stages_ms": {"k_sample": float(p[0]), "k_rollout": float(p[1]), "k_update": float(p[2])},
            "k_sample": dict(hbm_line(F.sample_bytes(K, Dp), float(p[0]), peaks),
                             note="issue-bound: a Philox call and two Box-Muller pairs per 16-byte store"),
            "k_update": hbm_line(F.update_bytes(K, Dp), float(p[2]), peaks)}


def multi_instance(peak, steps=20):
    """The persistent multi-instance launch (one kernel per control step for
    every instance): the 16-instance mix -- heightfield with the 0.3 m step box,
    K in {256 ... 4096}, H in {50, 100, 150} by seed 2 -- at the block shape the
    autotuner picks on it (128 threads x 3 blocks per SM), timed by CUDA events
    over back-to-back batch steps.  FLOPs: the flat-ground sub-step count, so the
    terrain's extra work is not credited."""
    from paper_2409_10469_gb300 import flops as F, multi, workloads as W
    r = multi.run(16, steps=steps, shapes=[(128, 3)], autotune=False)
    ms = r["ms_per_batch_step"]["128x3"]
    n_sub = W.config_terrain().mppi["n_sub"]
    fl = sum(F.rollout_flops(K, H, n_sub) for K, H in r["mix_K_H"])
    ach = fl / (ms * 1e-3) / 1e12
    return {"instances": 16, "shape": "128x3", "ms_per_batch_step": ms,
            "rollout_steps_per_batch_step": r["rollout_steps_per_batch_step"],
            "rollout_steps_per_s": r["best_rollout_steps_per_s"],
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "kernel": "k_batch<128, UNI_TERRAIN> (one model and cost: parameter-bank form)", "flops_per_launch": fl}}


def run_ours(args):
    import torch
    from paper_2409_10469_gb300 import _mppi, flops as F, workloads as W

    rank, world_size, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world_size > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    cfg = W.config_trot(K=K_BENCH, H=H_BENCH)
    m = dict(cfg.mppi)
    m["inst"] = rank        # independent instance per rank (own Philox stream)
    stream = torch.cuda.Stream()
    ctl = _mppi.Controller(cfg.robot, cfg.cost, m, stream=stream.cuda_stream, block=args.block)
    ctl.set_nominal(cfg.mu0)
    x0_d = torch.tensor(cfg.x0, dtype=torch.float32, device="cuda")
    u0_d = torch.empty(12, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    # clocks: one nvidia-smi stream from before the warm-up to the end of the run
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local_rank).start()

    # warm-up
    for s in range(args.warmup):
        ctl.step(x0_d, s, u0_out=u0_d)
    torch.cuda.synchronize()

    ctl.set_timing(False)            # the library's per-kernel events stay out of the timed steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_ms = []
    launches0 = ctl.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler.window():
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(s))          # evict L2 between steps (outside the events)
                starts[s].record(stream)
            ctl.step(x0_d, args.warmup + s, u0_out=u0_d)
            ends[s].record(stream)
            if (s + 1) % 16 == 0 or s == args.steps - 1:
                stream.synchronize()
            k_ms.append(None)
        torch.cuda.synchronize()
    # per-kernel times of every step: re-run with the library's events read per step
    ctl.set_timing(True)
    ker = []
    for s in range(min(args.steps, 64)):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        ctl.step(x0_d, args.warmup + args.steps + s, u0_out=u0_d)
        ker.append(ctl.timings())
    launches = ctl.launch_count() - launches0
    comp = component_ms(ctl, stream, flush, K_BENCH)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])
    mean_ms = float(step_ms.mean())
    from paper_2409_10469_gb300 import dist as D
    mean_ms = D.max_over_ranks(mean_ms, device="cuda")
    ker = np.array(ker)
    timed_launches = args.steps   # one kernel per step: sampling, rollouts, update (timed loop only)

    # end to end through the C ABI with host buffers (pinned x0 in, u0 out)
    x0_h = torch.tensor(cfg.x0, dtype=torch.float32).pin_memory()
    u0_h = torch.empty(12, dtype=torch.float32).pin_memory()
    e2e = []
    n_e2e = max(8, min(args.steps, 64))
    for s in range(3 + n_e2e):  # the first 3 calls warm the host buffers' path up, untimed
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        stream.synchronize()
        t = time.perf_counter()
        ctl.step(x0_h, 10000 + s, u0_out=u0_h)
        if s >= 3:
            e2e.append(time.perf_counter() - t)
    e2e_ms = float(np.mean(e2e)) * 1e3
    sampler.stop()
    clocks = sampler.summary()
    ctl.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    rollout_ms = float(ker[:, 1].mean())
    fl = F.rollout_flops(K_BENCH, H_BENCH, m["n_sub"])
    fl_dyn = F.rollout_flops(K_BENCH, H_BENCH, m["n_sub"], precise=False)
    achieved = fl / (rollout_ms * 1e-3) / 1e12
    sm_max = (peaks or {}).get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = F.fp32_peak_tflops(n_sm, sm_max)
    full_occ = full_occupancy_roofline(W.config_trot, F, flush, peak, n_sm)
    prop = proposal_form(flush)
    direct = direct_form(flush, peaks)
    multi16 = multi_instance(peak)
    value = D.job_throughput(K_BENCH * H_BENCH, world_size, mean_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "rollout-steps/s", "n_gpus": world_size,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(m["n_sub"]),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "max": float(step_ms.max())},
        # the step is one kernel: knot sampling, rollouts and the fused update (Eq. 1-2, shift)
        "kernel_ms": {"k_rollout": rollout_ms},
        # the noise and update kernels on their own calls (mppi_sample, mppi_update) at this K
        "roofline_aux": {"k_sample": hbm_line(F.sample_bytes(K_BENCH), comp["k_sample"], peaks),
                         "k_update": hbm_line(F.update_bytes(K_BENCH), comp["k_update"], peaks)},
        "roofline_full_occupancy": full_occ,
        # the learned-proposal form (K = 2048, half the samples around the network's mean)
        "proposal_form": prop,
        # direct targets (12 H sampled parameters per sample): sampler, rollouts, a three-launch update
        "direct_form": direct,
        # many controllers in one persistent launch per step (16 instances, uneven K and H)
        "multi_instance": multi16,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": rollout_traffic(),
                     "kernel": "k_rollout", "flops_per_launch": fl,
                     # the same time over the dynamics' FLOPs alone (plain FP32 contact geometry)
                     "dynamics_only": {"flops_per_launch": fl_dyn, "achieved": fl_dyn / (rollout_ms * 1e-3) / 1e12,
                                       "frac": fl_dyn / (rollout_ms * 1e-3) / 1e12 / peak},
                     "peak_source": "%d SMs (device properties) x 128 FP32 lanes x 2 x %.0f MHz "
                                    "(max SM clock, MEASURED_PEAKS.json)" % (n_sm, sm_max)},
        "e2e": {"value": world_size * K_BENCH * H_BENCH / (e2e_ms * 1e-3), "unit": "rollout-steps/s",
                "ms_per_step": e2e_ms, "p99_ms": float(np.percentile(np.array(e2e) * 1e3, 99)),
                "h2d_bytes_per_step": 4 * 37, "d2h_bytes_per_step": 4 * 12 + 4},
        "gpu_launches": timed_launches,
        "clocks": clocks,
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, seconds=args.cpu_seconds)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        import __graft_entry__ as g
        g.build()
        run_ours(args)


if __name__ == "__main__":
    main()
