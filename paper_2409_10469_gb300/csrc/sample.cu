// sample.cu -- K1: knot samples for Alg. 1's sampling step (arXiv 2409.10469,
// Sec. II-B: u ~ N(mu, Sigma), Sigma diagonal and fixed; Sec. III-B: the samples
// are the 4 spline knots of 12 joint targets).
//
// Noise per the model spec: Philox4x32-10 (Salmon et al., SC'11) with key = the
// 64-bit seed and counter (g, k, step, instance), g = 0..11; each call's 4 words
// give 4 normals by Box-Muller on word pairs.  The FP32 operation sequence (ln,
// sin/cos, the perturbation) is fixed so that it is bit-exact with any other
// implementation of the same spec: every rounding step is an explicit _rn
// intrinsic, so nvcc cannot contract or reorder it.
//
// One thread per (sample, Philox call): it writes 4 consecutive knots of one
// sample as a single 16-byte store, so a warp writes 512 contiguous bytes.
#include "kernels.h"

namespace mppi {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// ln(x) for a positive normal float: x = 2^e m, m in [sqrt(1/2), sqrt(2)],
// s = (m - 1)/(m + 1), ln m = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9),
// ln 2 split Cody-Waite style into 0x3f317200 + 0x35bfbe8e.
__device__ __forceinline__ float ln_spec(float x) {
    uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > __uint_as_float(0x3fb504f3u)) { m = __fmul_rn(m, 0.5f); e += 1; }
    float f = __fsub_rn(m, 1.0f);
    float s = __fdiv_rn(f, __fadd_rn(m, 1.0f));
    float z = __fmul_rn(s, s);
    float p = __fmaf_rn(z, __uint_as_float(0x3de38e39u), __uint_as_float(0x3e124925u));  // 1/9, 1/7
    p = __fmaf_rn(z, p, __uint_as_float(0x3e4ccccdu));                                  // 1/5
    p = __fmaf_rn(z, p, __uint_as_float(0x3eaaaaabu));                                  // 1/3
    p = __fmul_rn(p, z);
    float s2 = __fadd_rn(s, s);
    float r = __fmaf_rn(s2, p, s2);
    float ef = (float)e;
    return __fmaf_rn(ef, __uint_as_float(0x3f317200u), __fmaf_rn(ef, __uint_as_float(0x35bfbe8eu), r));
}

// cos and sin of 2 pi n 2^-24 (n 24-bit): exact quarter-turn reduction from the
// integer, x in [-pi/4, pi/4), Taylor polynomials to x^9 (sin) and x^10 (cos).
__device__ __forceinline__ void sincos2pi_spec(uint32_t n, float& c, float& s) {
    uint32_t qd = (n >> 22) & 3u;
    int32_t fr = (int32_t)(n & 0x3fffffu);
    if (fr >= 0x200000) { fr -= 0x400000; qd = (qd + 1u) & 3u; }
    float t = __fmul_rn((float)fr, 2.384185791015625e-07f);   // 2^-22, exact
    float xr = __fmul_rn(t, __uint_as_float(0x3fc90fdbu));     // pi / 2
    float x2 = __fmul_rn(xr, xr);
    float ps = __fmaf_rn(x2, __uint_as_float(0x3638ef1du), __uint_as_float(0xb9500d01u));  // 1/9!, -1/7!
    ps = __fmaf_rn(x2, ps, __uint_as_float(0x3c088889u));                                  // 1/5!
    ps = __fmaf_rn(x2, ps, __uint_as_float(0xbe2aaaabu));                                  // -1/3!
    float sn = __fmaf_rn(__fmul_rn(xr, x2), ps, xr);
    float pc = __fmaf_rn(x2, __uint_as_float(0xb493f27eu), __uint_as_float(0x37d00d01u));  // -1/10!, 1/8!
    pc = __fmaf_rn(x2, pc, __uint_as_float(0xbab60b61u));                                  // -1/6!
    pc = __fmaf_rn(x2, pc, __uint_as_float(0x3d2aaaabu));                                  // 1/4!
    pc = __fmaf_rn(x2, pc, -0.5f);
    float cs = __fmaf_rn(x2, pc, 1.0f);
    switch (qd) {
        case 0: c = cs; s = sn; break;
        case 1: c = -sn; s = cs; break;
        case 2: c = -cs; s = -sn; break;
        default: c = sn; s = -cs; break;
    }
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& e0, float& e1) {
    float u1 = __fmul_rn((float)((a >> 8) + 1u), 5.9604644775390625e-08f);   // 2^-24
    float l = ln_spec(u1);
    float r = __fsqrt_rn(__fmul_rn(-2.0f, l));
    float c, s;
    sincos2pi_spec(b >> 8, c, s);
    e0 = __fmul_rn(r, c);
    e1 = __fmul_rn(r, s);
}

__global__ void __launch_bounds__(256) k_sample(SampleArgs a) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = tid / (D / 4), g = tid % (D / 4);
    if (k >= a.K) return;
    const int kp0 = a.K - (a.mu_prop ? a.n_prop : 0);
    const bool prop = a.mu_prop && k >= kp0;
    const float* ctr = prop ? a.mu_prop : a.mu;
    float eps[4] = {0.f, 0.f, 0.f, 0.f};
    if (!(k == 0 || (prop && k == kp0))) {
        uint32_t c[4] = {(uint32_t)g, (uint32_t)k, a.step, a.inst};
        philox4x32_10(c, a.key0, a.key1);
        box_muller(c[0], c[1], eps[0], eps[1]);
        box_muller(c[2], c[3], eps[2], eps[3]);
    }
    float4 out;
    float* o = &out.x;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int d = 4 * g + i, jt = d % 3;
        float v = __fmaf_rn(a.sigma[d], eps[i], __ldg(ctr + d));
        o[i] = fminf(fmaxf(v, a.q_lo[jt]), a.q_hi[jt]);
    }
    reinterpret_cast<float4*>(a.U + (size_t)k * D)[g] = out;
}

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st) {
    if (a.K <= 0) return cudaSuccess;
    const long threads = (long)a.K * (D / 4);
    const int block = 256;
    k_sample<<<(int)((threads + block - 1) / block), block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
