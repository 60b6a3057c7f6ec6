"""K-sharded control step: one MPPI controller whose K samples are split over
several ranks (one process per GPU).

Alg. 1 treats its samples independently until Eq. 1, and Eq. 1's weights factor
as exp(-(L_k - L_min)/lambda) = exp(-(L_k - m_r)/lambda) exp(-(m_r - L_min)/lambda)
for any shard minimum m_r.  So each rank rolls out a contiguous range of the
step's samples (the same Philox stream: sample k is the same knot vector on
every rank), forms its partial sums around its own minimum (mppi_step_partial:
m_r, Z_r, S_r[48] in FP64), and two collectives finish the step:

  all-reduce(min) of m_r                     -> L_min
  all-reduce(sum) of exp(-(m_r - L_min)/lambda) (Z_r, S_r)   -> (Z, S)

after which every rank holds the same sums, and mppi_step_finalize gives every
rank the same mu' = S / Z, applied control and shifted nominal.  The two
collectives carry 1 + 49 doubles per control step.

The protocol is written against two reduction callables, so the same code runs
over torch.distributed (gloo on CPUs, NCCL on GPUs) or an in-process stand-in.
"""
from __future__ import annotations

import math

import numpy as np

from . import _mppi

N_SUMS = _mppi.SHARD_PARTIAL - 1   # Z and S[48]


def shard_range(K: int, rank: int, world: int):
    """(k0, n): rank's contiguous share of K samples; the first K % world ranks
    take one more, so the ranges tile 0..K-1 exactly (n may be 0 when world > K)."""
    if not (0 <= rank < world) or K < 0:
        raise ValueError("bad rank, world or K")
    base, extra = divmod(K, world)
    k0 = rank * base + min(rank, extra)
    return k0, base + (1 if rank < extra else 0)


def empty_partial() -> np.ndarray:
    """The partial of a rank without samples: no finite cost, zero sums."""
    p = np.zeros(_mppi.SHARD_PARTIAL, np.float64)
    p[0] = math.inf
    return p


def combine(part, lam: float, all_reduce_min, all_reduce_sum) -> np.ndarray:
    """This rank's partial (m, Z, S[48]) -> the sums (Z, S[48]) over every rank,
    relative to the global L_min (Eq. 1's factorisation; FP64 throughout).  A
    rank whose samples have no finite cost contributes zero."""
    part = np.asarray(part, np.float64)
    m = float(part[0])
    Lmin = float(all_reduce_min(m))
    f = math.exp(-(m - Lmin) / lam) if (math.isfinite(m) and math.isfinite(Lmin)) else 0.0
    return np.asarray(all_reduce_sum(f * part[1:]), np.float64)


def torch_reducers(group=None, device=None):
    """(all_reduce_min, all_reduce_sum) over a torch.distributed process group
    (float64 tensors on `device`: None for gloo's CPU tensors, a CUDA device for
    NCCL)."""
    import torch
    import torch.distributed as dist

    def rmin(v):
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
        return float(t.item())

    def rsum(a):
        t = torch.tensor(np.asarray(a, np.float64), device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()

    return rmin, rsum


def sharded_step(ctl, x0, step: int, rank: int, world: int, reducers, u0_out=None, mu_out=None):
    """One control step of `ctl` (a handle whose configuration, seed and nominal
    are the same on every rank) over its share of the K samples, finished by the
    two collectives of `reducers`; returns mppi_step_finalize's status (u0_out,
    mu_out as in mppi_step)."""
    k0, n = shard_range(ctl.K, rank, world)
    part = ctl.step_partial(x0, step, k0, n) if n > 0 else empty_partial()
    sums = combine(part, ctl.lam, *reducers)
    return ctl.step_finalize(sums, u0_out, mu_out, check=False)
