// update.cu -- K3/K4: softmax weights (Eq. 1), weighted mean (Eq. 2), applied
// control u = mu[0] and the receding-horizon shift (Alg. 1, last steps) of
// arXiv 2409.10469, Sec. II-B.
//
// One CTA of 512 threads (the step's tail is latency-bound: it reads n costs
// and n x 48 knots once).  L_min over finite costs; w_k = exp(-(L_k - L_min)/lambda)
// in FP32 (non-finite -> 0); the normaliser sum w is accumulated in FP64 (the
// only FP64 on the GPU path); the per-dimension sums sum w_k U_k use
// compensated (Kahan) FP32 per lane and an FP64 combine across warps.
#include "kernels.h"

namespace mppi {

constexpr int UPD_THREADS = 512;
constexpr int UPD_WARPS = UPD_THREADS / 32;

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= 3.402823466e38f; }

__global__ void __launch_bounds__(UPD_THREADS) k_update(UpdateArgs a) {
    __shared__ float s_min[UPD_WARPS];
    __shared__ double s_z[UPD_WARPS];
    __shared__ double s_part[UPD_WARPS][D];
    __shared__ float s_mu[D];
    __shared__ float s_lmin;
    __shared__ double s_Z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // L_min over finite costs
    float lm = INFINITY;
    for (int k = tid; k < a.n; k += UPD_THREADS) {
        float l = a.L[k];
        if (finitef(l)) lm = fminf(lm, l);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = fminf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if (lane == 0) s_min[warp] = lm;
    __syncthreads();
    if (tid == 0) {
        float v = s_min[0];
        for (int w = 1; w < UPD_WARPS; w++) v = fminf(v, s_min[w]);
        s_lmin = v;
    }
    __syncthreads();
    const float Lmin = s_lmin;
    const bool ok = finitef(Lmin);

    // normaliser Z = sum_k w_k in FP64
    double z = 0.0;
    if (ok)
        for (int k = tid; k < a.n; k += UPD_THREADS) {
            float l = a.L[k];
            if (finitef(l)) z += (double)expf(-(l - Lmin) * a.inv_lambda);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) s_z[warp] = z;

    // sum_k w_k U_k: warp w takes samples w, w + 16, ...; lane i < 24 owns dims 2i, 2i + 1
    float s0 = 0.f, s1 = 0.f, c0 = 0.f, c1 = 0.f;
    if (ok && lane < D / 2) {
        for (int k = warp; k < a.n; k += UPD_WARPS) {
            float l = __ldg(a.L + k);
            if (!finitef(l)) continue;
            float w = expf(-(l - Lmin) * a.inv_lambda);
            float2 u = __ldg(reinterpret_cast<const float2*>(a.U + (size_t)k * D) + lane);
            float y0 = w * u.x - c0, y1 = w * u.y - c1;
            float t0 = s0 + y0, t1 = s1 + y1;
            c0 = (t0 - s0) - y0; c1 = (t1 - s1) - y1;
            s0 = t0; s1 = t1;
        }
        s_part[warp][2 * lane] = (double)s0 - (double)c0;
        s_part[warp][2 * lane + 1] = (double)s1 - (double)c1;
    }
    __syncthreads();
    if (tid == 0) {
        double Z = 0.0;
        for (int w = 0; w < UPD_WARPS; w++) Z += s_z[w];
        s_Z = Z;
    }
    __syncthreads();
    if (tid < D) {
        float mu_new;
        if (ok) {
            double acc = 0.0;
            for (int w = 0; w < UPD_WARPS; w++) acc += s_part[w][tid];
            mu_new = (float)(acc / s_Z);
        } else {
            mu_new = a.mu[tid];  // every cost non-finite: keep the previous mean
        }
        s_mu[tid] = mu_new;
        if (a.mu_upd) a.mu_upd[tid] = mu_new;
        if (tid < NJ) a.u0[tid] = mu_new;  // the spline at tau = 0 is knot 0
    }
    if (tid == 0) {
        if (a.status) *a.status = ok ? 0 : 4;
        if (a.wsum) *a.wsum = s_Z;
    }
    __syncthreads();
    // shifted(mu): knot j re-sampled at tau_j + delta, held at tau = 1 past the end
    if (tid < D) {
        const int j = tid / NJ, i = tid % NJ;
        const float delta = a.H > 1 ? (float)a.ctrl_steps / (float)(a.H - 1) : 0.f;
        const float tau = fminf((float)j * (1.f / 3.f) + delta, 1.f);
        const float d0 = tau, d1 = tau - (1.f / 3.f), d2 = tau - (2.f / 3.f), d3 = tau - 1.f;
        const float B0 = d1 * d2 * d3 * -4.5f, B1 = d0 * d2 * d3 * 13.5f;
        const float B2 = d0 * d1 * d3 * -13.5f, B3 = d0 * d1 * d2 * 4.5f;
        a.mu[tid] = B0 * s_mu[i] + B1 * s_mu[NJ + i] + B2 * s_mu[2 * NJ + i] + B3 * s_mu[3 * NJ + i];
    }
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
    k_update<<<1, UPD_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
