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
    // sigma and the joint limits staged in shared memory: the lanes of a warp
    // index them at different places
    __shared__ float s_sig[D], s_lo[3], s_hi[3];
    if (threadIdx.x < D) s_sig[threadIdx.x] = a.sigma[threadIdx.x];
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = a.q_lo[threadIdx.x];
        s_hi[threadIdx.x] = a.q_hi[threadIdx.x];
    }
    __syncthreads();
    // (sample k, call g) = divmod(tid, G) by a multiply-high with floor(2^32 / G),
    // which is exact or one short, and one correction
    const uint32_t G = (uint32_t)a.Dp / 4;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t k = __umulhi(tid, a.g_magic), g = tid - k * G;
    if (g >= G) {
        k++;
        g -= G;
    }
    if (k >= (uint32_t)a.K) return;
    const uint32_t kp0 = (uint32_t)(a.K - (a.mu_prop ? a.n_prop : 0));
    const bool prop = a.mu_prop && k >= kp0;
    const float* ctr = prop ? a.mu_prop : a.mu;
    float eps[4] = {0.f, 0.f, 0.f, 0.f};
    if (!(k == 0 || (prop && k == kp0))) {
        uint32_t c[4] = {g, k, a.step, a.inst};
        philox4x32_10(c, a.key0, a.key1);
        box_muller(c[0], c[1], eps[0], eps[1]);
        box_muller(c[2], c[3], eps[2], eps[3]);
    }
    // parameter d = 4 g + i: joint (d mod 3) = (g + i) mod 3; sigma[d], or for
    // DIRECT sigma[d mod 12] = sigma[4 (g mod 3) + i]
    const uint32_t g3 = g % 3u;
    const uint32_t sb = a.interp == INTERP_DIRECT ? 4u * g3 : 4u * g;
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(ctr) + g);  // both means are 16-byte aligned
    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
    float4 out;
    float* o = &out.x;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t jt = g3 + i >= 3u ? g3 + i - 3u : g3 + i;
        float c = cv[i];
        if (prop && !(fabsf(c) <= 3.402823466e38f)) c = __ldg(a.mu + 4 * g + i);  // non-finite proposal: plain mean
        const float v = __fmaf_rn(s_sig[sb + i], eps[i], c);
        o[i] = fminf(fmaxf(v, s_lo[jt]), s_hi[jt]);
    }
    reinterpret_cast<float4*>(a.U + (size_t)k * a.Dp)[g] = out;
}

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st) {
    if (a.K <= 0) return cudaSuccess;
    const long G = a.Dp / 4;
    const long threads = (long)a.K * G;
    if (G < 2 || threads >= (1L << 32)) return cudaErrorInvalidValue;
    SampleArgs b = a;
    b.g_magic = (uint32_t)((1ull << 32) / (unsigned long long)G);
    const int block = 256;
    k_sample<<<(int)((threads + block - 1) / block), block, 0, st>>>(b);
    return cudaGetLastError();
}

// every 24-bit input of the Box-Muller pieces: the radius of word a = i << 8
// and the angle of word b = i << 8
__global__ void k_noise_tables(float* radius, float* cosv, float* sinv) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1u << 24)) return;
    radius[i] = box_muller_radius(i << 8);
    sincos2pi_spec(i, cosv[i], sinv[i]);
}

cudaError_t launch_noise_tables(float* radius, float* cosv, float* sinv, cudaStream_t st) {
    k_noise_tables<<<(1 << 24) / 256, 256, 0, st>>>(radius, cosv, sinv);
    return cudaGetLastError();
}

}  // namespace mppi
