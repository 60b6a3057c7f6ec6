"""Build libmppi_gb300.so (the C ABI of include/mppi.h) for sm_103a with nvcc.

Translation units are compiled in parallel and linked with nvcc -shared; the
library lands next to this file (in-tree, git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmppi_gb300.so")
SOURCES = ["api.cu", "sample.cu", "rollout.cu", "update.cu", "noalloc.cu", "batch.cu", "batch_uni.cu", "batch_uni_box.cu", "serve.cu", "mlp.cu", "gemm.cu", "features.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include"), "-I" + BUILD]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "mppi.h"))
    out.append(os.path.abspath(__file__))
    return out


TRIG_N = 512


def write_trig_table(path: str) -> None:
    """The precise sine / cosine table of csrc/precise.cuh: at a_j = j 2 pi / 512,
    (cos hi, cos lo, sin hi, sin lo) with hi the FP32 rounding of the double value
    and lo the FP32 rounding of the rest, as exact hexadecimal literals."""
    import math
    import struct

    def f32(x):
        return struct.unpack("f", struct.pack("f", x))[0]

    rows = []
    for j in range(TRIG_N):
        a = 2.0 * math.pi * j / TRIG_N
        c, s = math.cos(a), math.sin(a)
        ch, sh = f32(c), f32(s)
        vals = (ch, f32(c - ch), sh, f32(s - sh))
        rows.append("    {" + ", ".join("%sf" % float(v).hex() for v in vals) + "},")
    txt = ("// generated by build.py: sin / cos at j 2 pi / %d as FP32 pairs (do not edit)\n"
           "#pragma once\nnamespace mppi {\nconstexpr int TRIG_N = %d;\n"
           "static __device__ float4 g_trig[TRIG_N] = {\n%s\n};\n}  // namespace mppi\n"
           % (TRIG_N, TRIG_N, "\n".join(rows)))
    if os.path.exists(path) and open(path).read() == txt:
        return
    with open(path, "w") as f:
        f.write(txt)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    write_trig_table(os.path.join(BUILD, "trig_table.inc"))
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return LIB
    nvcc = _nvcc()

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        res = list(ex.map(one, SOURCES))
    if verbose:
        for _, log in res:
            sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in res] + ["-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
