"""CPU check of the tcgen05 encodings in csrc/tc.cuh before any kernel runs:
the shared-memory matrix descriptor and the BF16 x BF16 -> FP32 instruction
descriptor, field by field against the PTX ISA layout, and the core-matrix
tile offsets staying inside the staged tile."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include "tc.cuh"
using namespace mppi::tc;
int main() {
    printf("%llx\n", (unsigned long long)smem_desc(0x1230, 128, 1024));
    printf("%llx\n", (unsigned long long)smem_desc(0x2a400, 128, 1024));
    printf("%x\n", idesc_bf16_f32(128, 256));
    printf("%x\n", idesc_bf16_f32(128, 64));
    unsigned mx = 0;
    for (int r = 0; r < 256; r++) for (int k = 0; k < 64; k++) { unsigned o = tile_offset(r, k); if (o > mx) mx = o; }
    printf("%u\n", mx);
    printf("%u %u %u\n", tile_offset(0, 8), tile_offset(8, 0), tile_offset(1, 1));
    return 0;
}
'''


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    d = tmp_path_factory.mktemp("tc")
    src = d / "enc.cu"
    src.write_text(SRC)
    exe = d / "enc"
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_2409_10469_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return out


def field(v, lo, n):
    return (v >> lo) & ((1 << n) - 1)


def test_smem_descriptor_fields(values):
    for line, addr in ((values[0], 0x1230), (values[1], 0x2a400)):
        v = int(line, 16)
        assert field(v, 0, 14) == addr >> 4            # start address >> 4
        assert field(v, 16, 14) == 128 >> 4            # leading byte offset (K direction)
        assert field(v, 32, 14) == 1024 >> 4           # stride byte offset (8-row groups)
        assert field(v, 46, 3) == 0b001                # fixed constant
        assert field(v, 49, 3) == 0 and field(v, 52, 1) == 0   # base offset, LBO mode
        assert field(v, 61, 3) == 0                    # no swizzle
        assert field(v, 14, 2) == 0 and field(v, 30, 2) == 0 and field(v, 53, 8) == 0


def test_instruction_descriptor_fields(values):
    for line, n in ((values[2], 256), (values[3], 64)):
        v = int(line, 16)
        assert field(v, 0, 4) == 0                     # dense, no saturate
        assert field(v, 4, 2) == 1                     # D = F32
        assert field(v, 7, 3) == 1 and field(v, 10, 3) == 1   # A = B = BF16 (same type)
        assert field(v, 13, 2) == 0                    # no negation
        assert field(v, 15, 1) == 0 and field(v, 16, 1) == 0  # both K-major
        assert field(v, 17, 6) == n >> 3               # N / 8
        assert field(v, 23, 1) == 0
        assert field(v, 24, 5) == 128 >> 4             # M / 16
        assert field(v, 29, 3) == 0


def test_tile_offsets_stay_in_tile(values):
    assert int(values[4]) == 256 * 64 * 2 - 2          # last bf16 of a 256 x 64 tile
    lbo, sbo, elem = (int(x) for x in values[5].split())
    assert (lbo, sbo, elem) == (128, 1024, 18)
