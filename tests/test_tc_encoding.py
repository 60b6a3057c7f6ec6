"""CPU check of the tcgen05 encodings in csrc/tc.cuh before any kernel runs:
the shared-memory matrix descriptors (no swizzle, and the 128-byte swizzle a
TMA box of 64 bf16 per row writes) and the BF16 x BF16 -> FP32 instruction
descriptor, field by field against the PTX ISA layout, the core-matrix tile
offsets staying inside the staged tile, and the TMA-fed kernel's ring and
split-K arithmetic (gemm.cu) on the shapes the network uses."""
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
    printf("%llx\n", (unsigned long long)smem_desc_sw128(0x4400));
    printf("%llx\n", (unsigned long long)(smem_desc_sw128(0x4400) + 2 * 3));
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


def test_swizzled_descriptor_fields(values):
    v = int(values[6], 16)
    assert field(v, 0, 14) == 0x4400 >> 4              # start (1024-byte aligned tile)
    assert field(v, 16, 14) == 1                       # LBO unused by the swizzled K-major layout
    assert field(v, 32, 14) == 1024 >> 4               # 8 rows x 128 B per row group
    assert field(v, 46, 3) == 0b001
    assert field(v, 49, 3) == 0 and field(v, 52, 1) == 0
    assert field(v, 61, 3) == 2                        # 128-byte swizzle
    # the 4th 16-wide K slice starts 3 x 32 bytes in: only the start field moves
    w = int(values[7], 16)
    assert field(w, 0, 14) == (0x4400 + 96) >> 4 and (w >> 14) == (v >> 14)


def ring_plan(M, K, nsplit, grid, stages=4, ntiles=1):
    """The TMA kernel's schedule: (unit, k-chunk range) per CTA, the ring slot and
    phase of every chunk, and the last issue per slot its producer drains."""
    mtiles, nk = -(-M // 128), -(-K // 64)
    kcs = -(-nk // nsplit)
    assert (nsplit - 1) * kcs < nk
    units = mtiles * ntiles * nsplit
    plans = []
    for b in range(min(grid, units)):
        it, chunks = 0, []
        for u in range(b, units, grid):
            sp, nt, mt = u % nsplit, (u // nsplit) % ntiles, u // (nsplit * ntiles)
            assert mt < mtiles and nt < ntiles
            kb, ke = sp * kcs, min(nk, sp * kcs + kcs)
            assert kb < ke                               # no empty range
            for kc in range(kb, ke):
                chunks.append((it % stages, (it // stages) & 1, kc))
                it += 1
        last = {}
        for s in range(min(stages, it)):
            i = it - 1 - ((it - 1 - s) % stages)
            assert i % stages == s and i < it and i + stages >= it
            last[s] = i
        plans.append((chunks, last))
    return plans


@pytest.mark.parametrize("M,K,nsplit,grid,stages,ntiles", [
    (128, 64, 1, 148, 4, 1), (39013, 256, 1, 148, 3, 1), (256, 4096, 16, 148, 3, 1), (48, 65536, 64, 148, 4, 1),
    (300, 64, 1, 2, 4, 4), (256, 320, 2, 1, 3, 2), (16384, 256, 1, 152, 3, 2), (4096, 256, 1, 152, 4, 4)])
def test_tma_ring_schedule(M, K, nsplit, grid, stages, ntiles):
    for chunks, last in ring_plan(M, K, nsplit, grid, stages, ntiles):
        # every chunk coordinate is a whole 64-element (128-byte) step: TMA x alignment
        assert all(kc * 64 * 2 % 16 == 0 for _, _, kc in chunks)
        # consecutive uses of a slot alternate phase
        seen = {}
        for s, ph, _ in chunks:
            if s in seen:
                assert ph == seen[s] ^ 1
            seen[s] = ph


def test_split_choice_keeps_ranges_nonempty():
    """the host's split rule (gemm_tma_split) against the kernel's range rule:
    ranges of ceil(chunks / nsplit) chunks, none empty, at most 64 ranges, the
    work units within the SM count"""
    def split(M, K, sms=148, max_split=64):
        mtiles, nk = -(-M // 128), -(-K // 64)
        target = sms // mtiles
        if target <= 1 or max_split <= 1:
            return 1
        kcs = max(4, -(-nk // target))
        ns = -(-nk // kcs)
        if ns > max_split:
            kcs = -(-nk // max_split)
            ns = -(-nk // kcs)
        return max(ns, 1)
    for M in (48, 256):
        for B in (1, 7, 64, 129, 256, 300, 1000, 4096, 65536, 100000):
            ns = split(M, B)
            nk = -(-B // 64)
            kcs = -(-nk // ns)
            assert 1 <= ns <= 64 and (ns - 1) * kcs < nk
            assert -(-M // 128) * ns <= 148


def test_tile_width_rule():
    """gemm_tma_nt: the widest of 256 / 128 / 64 columns whose tile count fills
    the SMs, 64 when N <= 64; every choice covers N in at most 4 column tiles
    and the shared-memory plan of each width fits 227 KB"""
    def nt_rule(M, N, nsplit, sms=152):
        if N <= 64:
            return 64
        mt = -(-M // 128) * nsplit
        if mt * -(-N // 256) >= sms:
            return 256
        if mt * -(-N // 128) >= sms:
            return 128
        return 64
    assert nt_rule(65536, 256, 1) == 256 and nt_rule(16384, 256, 1) == 128
    assert nt_rule(4096, 256, 1) == 64 and nt_rule(300, 48, 1) == 64 and nt_rule(256, 256, 64) == 128
    for nt, stages, nbuf in ((256, 3, 1), (128, 3, 2), (64, 4, 2)):
        stage = 128 * 64 * 2 + nt * 64 * 2
        smem = stages * stage + 8 * nbuf * 8192 + 1024
        assert stage % 1024 == 0 and smem + 112 <= 232448, (nt, smem)
        assert 2 * nt <= 512                          # two accumulators in TMEM
