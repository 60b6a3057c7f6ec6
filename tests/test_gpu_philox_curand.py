"""Pin of the oracle's Philox4x32-10 (Salmon et al., SC'11) against an
independent implementation of the same generator: cuRAND's device generator
Philox4_32_10, run as a library (its header-only device API).

curand_init(seed, subsequence, offset) keys the generator with the 64-bit seed
and starts its 128-bit counter at (offset / 4 in the low 64 bits, subsequence in
the high 64 bits); each curand4 returns the 4-word block of the current counter
and steps the counter by one.  So, for offsets that are multiples of 4, the raw
words must equal the oracle's philox(ctr, key) with ctr = [o lo, o hi, s lo, s hi]
(o = offset / 4, s = subsequence) and key = [seed lo, seed hi], and the second
call's words philox(ctr + 1, key).  A wrong round constant, key schedule,
multiplier or word order in the oracle would fail this, while the statistical
pins of test_oracle_sampling.py could not see it."""
import os
import subprocess

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SRC = r'''
#include <cstdio>
#include <curand_kernel.h>
struct Case { unsigned long long seed, sub, off; };
__global__ void draw(const Case* c, int n, uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(c[i].seed, c[i].sub, c[i].off, &st);
    out[2 * i] = curand4(&st);
    out[2 * i + 1] = curand4(&st);
}
int main() {
    int n = 0;
    if (scanf("%d", &n) != 1 || n < 1 || n > 4096) return 2;
    Case* h = new Case[n];
    for (int i = 0; i < n; i++)
        if (scanf("%llu %llu %llu", &h[i].seed, &h[i].sub, &h[i].off) != 3) return 2;
    Case* d = nullptr;
    uint4* o = nullptr;
    if (cudaMalloc(&d, n * sizeof(Case)) != cudaSuccess || cudaMalloc(&o, 2 * n * sizeof(uint4)) != cudaSuccess) return 3;
    cudaMemcpy(d, h, n * sizeof(Case), cudaMemcpyHostToDevice);
    draw<<<(n + 127) / 128, 128>>>(d, n, o);
    uint4* r = new uint4[2 * n];
    if (cudaMemcpy(r, o, 2 * n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    for (int i = 0; i < 2 * n; i++) printf("%u %u %u %u\n", r[i].x, r[i].y, r[i].z, r[i].w);
    cudaFree(d);
    cudaFree(o);
    return 0;
}
'''

M32 = 0xFFFFFFFF


# the sampler's counters (c0 = Philox call g, c1 = sample k, c2 = control step,
# c3 = instance): (seed, g, k, step, inst)
SAMPLER = [(0xDEADBEEF12345678, 5, 1000, 77, 3), (0, 0, 0, 0, 0), (2, 11, 4095, 123456, 63)]


def sampler_case(seed, g, k, step, inst):
    return seed, step + (inst << 32), 4 * (g + (k << 32))


def cases():
    rng = np.random.default_rng(20240916)
    seeds = [0, 1, 0xDEADBEEF12345678, (1 << 64) - 1, 42]
    subs = [0, 1, (1 << 32) + 5, (1 << 64) - 2]
    offs = [0, 4, 4 * ((1 << 32) - 1), 4 * (1 << 32) + 8]
    out = [(s, q, o) for s in seeds for q in subs for o in offs]
    for _ in range(200):
        out.append((int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2)), int(rng.integers(0, 1 << 63)),
                    4 * int(rng.integers(0, 1 << 60))))
    return out + [sampler_case(*c) for c in SAMPLER]


def oracle_blocks(seed, sub, off):
    o = off // 4
    ctr = [o & M32, (o >> 32) & M32, sub & M32, (sub >> 32) & M32]
    key = [seed & M32, (seed >> 32) & M32]
    first = O.philox(ctr, key)
    # the 128-bit counter plus one
    c = ctr[:]
    for w in range(4):
        c[w] = (c[w] + 1) & M32
        if c[w] != 0:
            break
    return first, O.philox(c, key)


@pytest.fixture(scope="module")
def curand_words(tmp_path_factory):
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    d = tmp_path_factory.mktemp("curand")
    (d / "draw.cu").write_text(SRC)
    exe = d / "draw"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", str(d / "draw.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    cs = cases()
    inp = "%d\n" % len(cs) + "".join("%d %d %d\n" % c for c in cs)
    res = subprocess.run([str(exe)], input=inp, check=True, capture_output=True, text=True).stdout.split("\n")
    words = np.array([[int(x) for x in line.split()] for line in res if line.strip()], dtype=np.uint64)
    assert words.shape == (2 * len(cs), 4)
    return cs, words


def test_philox_raw_words_equal_curand(curand_words):
    cs, words = curand_words
    for i, (seed, sub, off) in enumerate(cs):
        first, second = oracle_blocks(seed, sub, off)
        assert np.array_equal(first.astype(np.uint64), words[2 * i]), (seed, sub, off)
        assert np.array_equal(second.astype(np.uint64), words[2 * i + 1]), (seed, sub, off)


def test_sampler_counter_layout_matches_curand(curand_words):
    """the sampler's own counters are reached by cuRAND with offset = 4 (g + 2^32 k)
    and subsequence = step + 2^32 inst: the oracle's block for them equals cuRAND's"""
    cs, words = curand_words
    for c in SAMPLER:
        seed, g, k, step, inst = c
        i = cs.index(sampler_case(*c))
        got = O.philox([g, k, step, inst], [seed & M32, seed >> 32])
        assert np.array_equal(got.astype(np.uint64), words[2 * i]), c
