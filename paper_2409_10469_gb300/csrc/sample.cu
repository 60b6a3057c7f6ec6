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
// One thread per (sample, Philox call): it writes 4 consecutive parameters of
// one sample as a single 16-byte store, so a warp writes 512 contiguous bytes.
// Knot representations: 12 calls per sample (48 knots); DIRECT: 3 H calls (one
// 12-joint target per dt step, joint i perturbed with sigma[i]).
#include "kernels.h"
#include "noise.cuh"

namespace mppi {

__global__ void __launch_bounds__(256) k_sample(SampleArgs a) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int G = a.Dp / 4;
    const int k = tid / G, g = tid % G;
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
        float c = __ldg(ctr + d);
        if (prop && !(fabsf(c) <= 3.402823466e38f)) c = __ldg(a.mu + d);  // non-finite proposal: plain mean
        const float sg = a.interp == INTERP_DIRECT ? a.sigma[d % NJ] : a.sigma[d];
        float v = __fmaf_rn(sg, eps[i], c);
        o[i] = fminf(fmaxf(v, a.q_lo[jt]), a.q_hi[jt]);
    }
    reinterpret_cast<float4*>(a.U + (size_t)k * a.Dp)[g] = out;
}

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st) {
    if (a.K <= 0) return cudaSuccess;
    const long threads = (long)a.K * (a.Dp / 4);
    const int block = 256;
    k_sample<<<(int)((threads + block - 1) / block), block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
