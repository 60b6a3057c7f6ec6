"""Build the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Only tests/, __graft_entry__ (build, smoke) and bench.py's CPU-baseline legs
use the oracle; the product path never loads it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["dynamics.c", "world.c", "mppi.c"]
LIB = os.path.join(HERE, "liboracle.so")

# -ffp-contract=off: no implicit fused multiply-add, so the FP32 sampling
# sequence is exactly the one written (explicit fmaf) on every host.
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
          "-ffp-contract=off", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + srcs + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))


def build_variant(real: str = "float") -> str:
    """The same oracle source with `real` = float (an FP32 reference for
    measuring how much FP32 rounding alone moves a result)."""
    out = os.path.join(HERE, "liboracle_%s.so" % real)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h")]
    if os.path.exists(out) and all(os.path.getmtime(d) <= os.path.getmtime(out) for d in deps):
        return out
    cmd = ["gcc"] + CFLAGS + ["-DOR_REAL=" + real, "-Wno-double-promotion"] + srcs + ["-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build_count() -> str:
    """The same oracle source compiled as C++ with `real` = an operation-counting
    scalar (opcount.h): it measures how many floating-point operations the
    oracle's plain formulation performs."""
    out = os.path.join(HERE, "liboracle_count.so")
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, f) for f in ("oracle.h", "opcount.h", "opcount.cpp")]
    if os.path.exists(out) and all(os.path.getmtime(d) <= os.path.getmtime(out) for d in deps):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = (["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-x", "c++",
            "-include", os.path.join(HERE, "opcount.h"), "-DOR_REAL=or_creal"] + srcs
           + [os.path.join(HERE, "opcount.cpp"), "-o", tmp, "-lm"])
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out
