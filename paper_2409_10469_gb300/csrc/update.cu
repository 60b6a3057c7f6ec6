// update.cu -- K3/K4: softmax weights (Eq. 1), weighted mean (Eq. 2), applied
// control u = mu[0] and the receding-horizon shift (Alg. 1, last steps) of
// arXiv 2409.10469, Sec. II-B.
//
// G CTAs split the n samples into contiguous chunks.  Every CTA first takes
// L_min over all n costs (finite only; 4 B per sample, L2-resident), then for
// its chunk the FP32 weights w_k = exp(-(L_k - L_min)/lambda) (0 if L_k is not
// finite), their sum in FP64 (the normaliser: the only FP64 on the GPU path) and
// the per-dimension sums sum_k w_k U_k (compensated FP32 per lane, FP64 across
// warps).  Each CTA writes its 49 partial sums to scratch and bumps a counter;
// the CTA that sees the counter reach G - 1 (no waiting: it is simply the last
// to finish) adds the partials in CTA order -- so the result does not depend on
// scheduling -- forms mu' = S / Z, writes u0 = mu'[knot 0], the shifted nominal,
// the status, and re-arms the counter for the next launch.
#include "kernels.h"

namespace mppi {

constexpr int UPD_THREADS = 256;
constexpr int UPD_WARPS = UPD_THREADS / 32;

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= 3.402823466e38f; }

__global__ void __launch_bounds__(UPD_THREADS) k_update(UpdateArgs a) {
    __shared__ float s_min[UPD_WARPS];
    __shared__ double s_z[UPD_WARPS];
    __shared__ double s_part[UPD_WARPS][D];
    __shared__ float s_mu[D];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;

    // L_min over all finite costs
    float lm = INFINITY;
    for (int k = tid; k < a.n; k += UPD_THREADS) {
        float l = __ldg(a.L + k);
        if (finitef(l)) lm = fminf(lm, l);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = fminf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if (lane == 0) s_min[warp] = lm;
    __syncthreads();
    float Lmin = s_min[0];
#pragma unroll
    for (int w = 1; w < UPD_WARPS; w++) Lmin = fminf(Lmin, s_min[w]);
    const bool ok = finitef(Lmin);

    // this CTA's chunk
    const int chunk = (a.n + G - 1) / G;
    const int k0 = b * chunk, k1 = min(a.n, k0 + chunk);
    // normaliser partial (FP64)
    double z = 0.0;
    if (ok)
        for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
            float l = __ldg(a.L + k);
            if (finitef(l)) z += (double)expf(-(l - Lmin) * a.inv_lambda);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) s_z[warp] = z;
    // sum_k w_k U_k: warp w takes k0 + w, k0 + w + 8, ...; lane i < 24 owns dims 2i, 2i + 1
    float s0 = 0.f, s1 = 0.f, c0 = 0.f, c1 = 0.f;
    if (ok && lane < D / 2) {
        for (int k = k0 + warp; k < k1; k += UPD_WARPS) {
            float l = __ldg(a.L + k);
            float w = finitef(l) ? expf(-(l - Lmin) * a.inv_lambda) : 0.f;
            float2 u = __ldg(reinterpret_cast<const float2*>(a.U + (size_t)k * D) + lane);
            float y0 = w * u.x - c0, y1 = w * u.y - c1;
            float t0 = s0 + y0, t1 = s1 + y1;
            c0 = (t0 - s0) - y0;
            c1 = (t1 - s1) - y1;
            s0 = t0;
            s1 = t1;
        }
    }
    if (lane < D / 2) {
        s_part[warp][2 * lane] = (double)s0 - (double)c0;
        s_part[warp][2 * lane + 1] = (double)s1 - (double)c1;
    }
    __syncthreads();
    if (tid <= D) {
        double acc = 0.0;
        if (tid < D)
            for (int w = 0; w < UPD_WARPS; w++) acc += s_part[w][tid];
        else
            for (int w = 0; w < UPD_WARPS; w++) acc += s_z[w];
        a.part[(size_t)b * (D + 1) + tid] = acc;
    }
    // publish the partials, then count this CTA in
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last CTA: combine in CTA order, apply, shift
    if (tid < D) {
        float mu_new;
        if (ok) {
            double S = 0.0, Z = 0.0;
            for (int g = 0; g < G; g++) {
                S += __ldcg(a.part + (size_t)g * (D + 1) + tid);
                Z += __ldcg(a.part + (size_t)g * (D + 1) + D);
            }
            mu_new = (float)(S / Z);
            if (tid == 0 && a.wsum) *a.wsum = Z;
        } else {
            mu_new = a.mu[tid];  // every cost non-finite: keep the previous mean
        }
        s_mu[tid] = mu_new;
        if (a.mu_upd) a.mu_upd[tid] = mu_new;
        if (tid < NJ) a.u0[tid] = mu_new;  // the spline at tau = 0 is knot 0
    }
    if (tid == 0) {
        if (a.status) *a.status = ok ? 0 : 4;
        *a.counter = 0u;  // re-arm for the next launch (kernels on one stream are ordered)
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

int update_grid(int n) {
    int g = (n + 63) / 64;  // ~64 samples per CTA
    return g < 1 ? 1 : (g > UPDATE_MAX_CTAS ? UPDATE_MAX_CTAS : g);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
    k_update<<<update_grid(a.n), UPD_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
