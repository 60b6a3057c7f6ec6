// update.cu -- K3/K4: softmax weights (Eq. 1), weighted mean (Eq. 2), applied
// control u = mu[0] and the receding-horizon shift (Alg. 1, last steps) of
// arXiv 2409.10469, Sec. II-B.
//
// G CTAs split the n samples into contiguous chunks (a second grid dimension T
// tiles the 12 H parameters of direct targets into groups of 48; the knot
// representations have one tile and their own kernel).  Every CTA first takes
// L_min over all n costs (finite only; 4 B per sample, L2-resident), then for
// its chunk the FP32 weights w_k = exp(-(L_k - L_min)/lambda) (0 if L_k is not
// finite), their sum in FP64 (the normaliser: the only FP64 on the GPU path)
// and the sums sum_k w_k U_k of its 48 parameters (compensated FP32 per lane,
// FP64 across warps).  Each CTA writes its partial sums to scratch and bumps a
// counter; the CTA that sees the counter reach the grid size - 1 (no waiting:
// it is simply the last to finish) adds the partials in CTA order -- so the
// result does not depend on scheduling -- forms mu' = S / Z, writes u0 = the
// controls of step 0 (knot 0, or the first direct target), the shifted
// nominal, the status, and re-arms the counter for the next launch.
#include "kernels.h"

namespace mppi {

constexpr int UPD_THREADS = 256;
constexpr int UPD_WARPS = UPD_THREADS / 32;
constexpr int UPD_TILE = D;   // parameters per dimension tile

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= 3.402823466e38f; }

// One warp's share of a CTA chunk: samples k = kb, kb + UPD_WARPS, ... < ke, the
// lane's parameter pair u2[k * row2] weighted by w_k = exp(-(L_k - L_min) / lambda)
// (0 for a non-finite cost) into compensated (Kahan) sums, one sample at a time
// in order; the loads of 8 samples are issued together (one L2 round trip each)
__device__ __forceinline__ void sum_chunk(const float* L, const float2* u2, int row2, int kb, int ke, float Lmin,
                                          float inv_lambda, float& s0, float& s1, float& c0, float& c1) {
    constexpr int NB = 8;
    for (int kk = kb; kk < ke; kk += NB * UPD_WARPS) {
        float lb[NB];
        float2 ub[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int k = kk + q * UPD_WARPS;
            lb[q] = k < ke ? __ldg(L + k) : 0.f;
            ub[q] = k < ke ? __ldg(u2 + (size_t)k * row2) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            if (kk + q * UPD_WARPS >= ke) break;
            const float l = lb[q];
            const float w = finitef(l) ? expf(-(l - Lmin) * inv_lambda) : 0.f;
            const float2 u = ub[q];
            float y0 = w * u.x - c0, y1 = w * u.y - c1;
            float t0 = s0 + y0, t1 = s1 + y1;
            c0 = (t0 - s0) - y0;
            c1 = (t1 - s1) - y1;
            s0 = t0;
            s1 = t1;
        }
    }
}

// Knot representations (48 parameters): one parameter tile.
__global__ void __launch_bounds__(UPD_THREADS) k_update_knots(UpdateArgs a) {
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
    if (ok && lane < D / 2)
        sum_chunk(a.L, reinterpret_cast<const float2*>(a.U) + lane, D / 2, k0 + warp, k1, Lmin, a.inv_lambda, s0, s1,
                  c0, c1);
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
    // shifted(mu): the representation's interpolant re-sampled at tau_j + delta,
    // held at tau = 1 past the end
    if (tid < D) a.mu[tid] = shifted_knot(s_mu, a.interp, a.H, a.ctrl_steps, tid / NJ, tid % NJ);
}

// Direct targets (12 H parameters): G x T CTAs, T = ceil(12 H / 48) parameter tiles.
__global__ void __launch_bounds__(UPD_THREADS) k_update_tiled(UpdateArgs a) {
    __shared__ float s_min[UPD_WARPS];
    __shared__ double s_z[UPD_WARPS];
    __shared__ double s_part[UPD_WARPS][UPD_TILE];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x, T = gridDim.y, y = blockIdx.y;
    const int Dp = a.Dp, d0 = y * UPD_TILE;

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
    // normaliser partial (FP64), tile 0
    double z = 0.0;
    if (ok && y == 0)
        for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
            float l = __ldg(a.L + k);
            if (finitef(l)) z += (double)expf(-(l - Lmin) * a.inv_lambda);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) s_z[warp] = z;
    // sum_k w_k U_k: warp w takes k0 + w, k0 + w + 8, ...; lane i < 24 owns
    // parameters d0 + 2i, d0 + 2i + 1 (Dp is even, so a pair never straddles the end)
    const bool own = lane < UPD_TILE / 2 && d0 + 2 * lane < Dp;
    float s0 = 0.f, s1 = 0.f, c0 = 0.f, c1 = 0.f;
    if (ok && own)
        sum_chunk(a.L, reinterpret_cast<const float2*>(a.U + d0) + lane, Dp / 2, k0 + warp, k1, Lmin, a.inv_lambda, s0,
                  s1, c0, c1);
    if (lane < UPD_TILE / 2) {
        s_part[warp][2 * lane] = (double)s0 - (double)c0;
        s_part[warp][2 * lane + 1] = (double)s1 - (double)c1;
    }
    __syncthreads();
    if (tid < UPD_TILE && d0 + tid < Dp) {
        double acc = 0.0;
        for (int w = 0; w < UPD_WARPS; w++) acc += s_part[w][tid];
        a.part[(size_t)b * (Dp + 1) + d0 + tid] = acc;
    }
    if (y == 0 && tid == UPD_TILE) {
        double acc = 0.0;
        for (int w = 0; w < UPD_WARPS; w++) acc += s_z[w];
        a.part[(size_t)b * (Dp + 1) + Dp] = acc;
    }
    // publish the partials, then count this CTA in
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.counter, 1u) == (unsigned)(G * T - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last CTA: combine in CTA order (each thread's normaliser alongside its first
    // parameter), apply, shift
    double Z = 0.0;
    for (int d = tid; d < Dp; d += UPD_THREADS) {
        float mu_new;
        if (ok) {
            double S = 0.0;
            if (d == tid) {
                for (int g = 0; g < G; g++) {
                    S += __ldcg(a.part + (size_t)g * (Dp + 1) + d);
                    Z += __ldcg(a.part + (size_t)g * (Dp + 1) + Dp);
                }
            } else {
                for (int g = 0; g < G; g++) S += __ldcg(a.part + (size_t)g * (Dp + 1) + d);
            }
            mu_new = (float)(S / Z);
        } else {
            mu_new = a.mu[d];  // every cost non-finite: keep the previous mean
        }
        a.mu_upd[d] = mu_new;
        if (d < NJ) a.u0[d] = mu_new;  // the controls of step 0: the first direct target
    }
    if (tid == 0) {
        if (ok && a.wsum) *a.wsum = Z;  // thread 0 always owns parameter 0
        if (a.status) *a.status = ok ? 0 : 4;
        *a.counter = 0u;  // re-arm for the next launch (kernels on one stream are ordered)
    }
    __syncthreads();
    // direct targets move ctrl_steps steps earlier, the last one held (mu_upd was
    // written by this CTA before the barrier)
    for (int d = tid; d < Dp; d += UPD_THREADS) {
        const int t = d / NJ, i = d % NJ;
        const int src = min(t + a.ctrl_steps, a.H - 1);
        a.mu[d] = a.mu_upd[src * NJ + i];
    }
}

int update_grid(int n) {
    int g = (n + 127) / 128;  // ~128 samples per CTA (measured: 64 per CTA costs 3 us more at n = 4096)
    return g < 1 ? 1 : (g > UPDATE_MAX_CTAS ? UPDATE_MAX_CTAS : g);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
    if (a.Dp % 2 != 0 || a.Dp < D || (a.Dp > D && !a.mu_upd)) return cudaErrorInvalidValue;
    if (a.Dp == D) {
        k_update_knots<<<update_grid(a.n), UPD_THREADS, 0, st>>>(a);
    } else {
        const dim3 grid(update_grid(a.n), (a.Dp + UPD_TILE - 1) / UPD_TILE);
        k_update_tiled<<<grid, UPD_THREADS, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mppi
