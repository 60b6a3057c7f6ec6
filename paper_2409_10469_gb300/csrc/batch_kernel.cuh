// batch_kernel.cuh -- device side of the persistent multi-instance step
// (batch.cu): in-kernel sampling, the per-instance update in one block, and the
// kernel itself.  Included by batch.cu (the general kernel) and batch_uni.cu
// (its specialisation for launches whose instances share one model and cost),
// so the two compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "batch.cuh"
#include "noise.cuh"
#include "rollout.cuh"

namespace mppi {

// this lane's 12 knots of sample k (the leg's 3 joints at the 4 knots), and
// write them to U[k]; the same formula as k_sample, element by element
__device__ __forceinline__ void sample_lane(const InstDesc& d, int k, int leg, uint32_t step, bool write,
                                            float (&Uk)[NKNOT][3]) {
    const int kp0 = d.K - (d.mu_prop ? d.n_prop : 0);
    const bool prop = d.mu_prop && k >= kp0;
    const float* ctr = prop ? d.mu_prop : d.mu;
    const bool nominal = (k == 0) || (prop && k == kp0);
#pragma unroll
    for (int j = 0; j < NKNOT; j++) {
        float epsv[3];
        knot_normals(d.key0, d.key1, step, d.inst_id, (uint32_t)k, j * NJ + 3 * leg, epsv);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int dd = j * NJ + 3 * leg + i;
            const float eps = nominal ? 0.f : epsv[i];
            float c = __ldcg(ctr + dd);
            if (prop && !(fabsf(c) <= 3.402823466e38f)) c = __ldcg(d.mu + dd);  // non-finite proposal: plain mean
            float v = __fmaf_rn(d.sigma[dd], eps, c);
            v = fminf(fmaxf(v, d.q_lo[i]), d.q_hi[i]);
            Uk[j][i] = v;
            if (write) d.U[(size_t)k * D + dd] = v;
        }
    }
}

__device__ __forceinline__ bool finite_f(float x) { return fabsf(x) <= 3.402823466e38f; }

// Eq. 1, Eq. 2, apply, shift for one instance in one block.  The weights
// exp(-(L_k - L_min) / lambda) are computed once per sample -- exponent and exp
// in FP64, kept as FP32 pairs (about 48 significant bits) -- for sub-chunks of
// UPD_SUB samples in shared memory; the sums run over 8 fixed groups of samples
// (k = g mod 8, each in increasing k) whatever the block size, as float-float
// pairs (the products' rounding errors by FMA), and are combined in group order:
// the result does not depend on the block shape or on the other instances in
// the launch.
constexpr int UPD_GROUPS = 8;
constexpr int UPD_SUB = 256;  // a multiple of UPD_GROUPS: every group keeps its order across sub-chunks

// (s, e) += (v, ve): s + v split exactly into the new s and an error term
// (Knuth's TwoSum), the error and the low parts into e
__device__ __forceinline__ void bu_ff_add(float& s, float& e, float v, float ve) {
    // _rn intrinsics: never contracted with a preceding product (which would break TwoSum)
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    e = __fadd_rn(e, __fadd_rn(ve, err));
}

template <int BLOCK>
__device__ void block_update(const InstDesc& d, float* u0_row) {
    constexpr int W = BLOCK / 32;
    constexpr int ACTIVE = BLOCK / 12;  // groups processed at once (12 lanes each, four dims per lane)
    constexpr int GPT = (UPD_GROUPS + ACTIVE - 1) / ACTIVE;  // groups per thread
    __shared__ float s_min[W];
    __shared__ float2 s_z[UPD_GROUPS];
    __shared__ float2 s_part[UPD_GROUPS][D];
    __shared__ float s_mu[D];
    __shared__ float2 s_w[UPD_SUB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = d.K;
    float lm = INFINITY;
    for (int k = tid; k < K; k += BLOCK) {
        float l = __ldcg(d.L + k);
        if (finite_f(l)) lm = fminf(lm, l);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = fminf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if (lane == 0) s_min[warp] = lm;
    __syncthreads();
    float Lmin = s_min[0];
#pragma unroll
    for (int w = 1; w < W; w++) Lmin = fminf(Lmin, s_min[w]);
    const bool ok = finite_f(Lmin);
    const int li = tid % 12;
    const bool grp = tid < ACTIVE * 12;
    float sh[GPT][4], se[GPT][4], zh[GPT], ze[GPT];
#pragma unroll
    for (int gi = 0; gi < GPT; gi++) {
        zh[gi] = 0.f;
        ze[gi] = 0.f;
#pragma unroll
        for (int e = 0; e < 4; e++) { sh[gi][e] = 0.f; se[gi][e] = 0.f; }
    }
    if (ok)
        for (int kb = 0; kb < K; kb += UPD_SUB) {
            const int ke = min(K, kb + UPD_SUB);
            __syncthreads();  // the previous sub-chunk's weights are consumed
            for (int i = tid; i < UPD_SUB; i += BLOCK) {
                const int k = kb + i;
                float2 wk = make_float2(0.f, 0.f);
                if (k < ke) {
                    const float l = __ldcg(d.L + k);
                    if (finite_f(l)) {
                        const double wd = exp(-((double)l - (double)Lmin) * d.inv_lambda);
                        wk.x = (float)wd;
                        wk.y = (float)(wd - (double)wk.x);
                    }
                }
                s_w[i] = wk;
            }
            __syncthreads();
#pragma unroll
            for (int gi = 0; gi < GPT; gi++) {
                const int g = tid / 12 + gi * ACTIVE;
                if (!grp || g >= UPD_GROUPS) continue;
                // samples g, g + 8, ... of the sub-chunk in order; the loads of 8
                // of them are issued together (one L2 round trip per 8 samples)
                constexpr int NB = 8;
                for (int k0 = kb + g; k0 < ke; k0 += NB * UPD_GROUPS) {
                    float4 ub[NB];
#pragma unroll
                    for (int q = 0; q < NB; q++) {
                        const int k = k0 + q * UPD_GROUPS;
                        ub[q] = k < ke ? __ldcg(reinterpret_cast<const float4*>(d.U + (size_t)k * D) + li)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < NB; q++) {
                        const int k = k0 + q * UPD_GROUPS;
                        if (k >= ke) break;
                        const float2 wk = s_w[k - kb];
                        bu_ff_add(zh[gi], ze[gi], wk.x, wk.y);
                        const float u[4] = {ub[q].x, ub[q].y, ub[q].z, ub[q].w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const float pr = wk.x * u[e];
                            bu_ff_add(sh[gi][e], se[gi][e], pr, fmaf(wk.y, u[e], fmaf(wk.x, u[e], -pr)));
                        }
                    }
                }
            }
        }
#pragma unroll
    for (int gi = 0; gi < GPT; gi++) {
        const int g = tid / 12 + gi * ACTIVE;
        if (!grp || g >= UPD_GROUPS) continue;
#pragma unroll
        for (int e = 0; e < 4; e++) s_part[g][4 * li + e] = make_float2(sh[gi][e], se[gi][e]);
        if (li == 0) s_z[g] = make_float2(zh[gi], ze[gi]);
    }
    __syncthreads();
    if (tid < D) {
        float mu_new;
        if (ok) {
            // the groups' pairs added in order, float-float (FP32 pipe), then the quotient
            float sh0 = s_part[0][tid].x, se0 = s_part[0][tid].y, zh0 = s_z[0].x, ze0 = s_z[0].y;
            for (int q = 1; q < UPD_GROUPS; q++) {
                bu_ff_add(sh0, se0, s_part[q][tid].x, s_part[q][tid].y);
                bu_ff_add(zh0, ze0, s_z[q].x, s_z[q].y);
            }
            mu_new = ff_div(make_float2(sh0, se0), make_float2(zh0, ze0));
        } else {
            mu_new = __ldcg(d.mu + tid);
        }
        s_mu[tid] = mu_new;
        d.mu_upd[tid] = mu_new;
        if (tid < NJ) {
            d.u0[tid] = mu_new;
            u0_row[tid] = mu_new;
        }
    }
    if (tid == 0) *d.status = ok ? 0 : 4;
    __syncthreads();
    if (tid < D) d.mu[tid] = shifted_knot(s_mu, d.interp, d.H, d.ctrl_steps, tid / NJ, tid % NJ);
}

// Kernel variants: UNI_NONE reads each item's model and cost from its
// descriptor; the UNI_* forms serve launches whose instances share one model
// and cost (the launch parameters), one per terrain / box combination, so each
// holds only the rollout code its model runs.
enum : int { UNI_NONE = 0, UNI_FLAT = 1, UNI_TERRAIN = 2, UNI_FLAT_BOX = 3, UNI_TERRAIN_BOX = 4 };

// the shared-model variant for a model
inline int uni_kind(const DevModel& m) {
    const bool terr = m.terrain != 0 || m.n_sbox > 0;
    return m.has_box ? (terr ? UNI_TERRAIN_BOX : UNI_FLAT_BOX) : (terr ? UNI_TERRAIN : UNI_FLAT);
}

// one item's rollouts on the terrain / box variant its model needs
template <int UNI>
__device__ __forceinline__ float rollout_item(const DevModel& m, const DevCost& c, const HorizonArgs& hz,
                                              const float* x0, const float (&Uk)[NKNOT][3], int leg, int k,
                                              bool valid) {
    if (UNI == UNI_FLAT) return rollout_lane<0, false>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
    if (UNI == UNI_TERRAIN) return rollout_lane<1, false>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
    if (UNI == UNI_FLAT_BOX) return rollout_lane<0, true>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
    if (UNI == UNI_TERRAIN_BOX) return rollout_lane<1, true>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
    if (m.terrain != 0 || m.n_sbox > 0)
        return m.has_box ? rollout_lane<1, true>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr)
                         : rollout_lane<1, false>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
    return m.has_box ? rollout_lane<0, true>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr)
                     : rollout_lane<0, false>(m, c, hz, x0, Uk, nullptr, leg, k, valid, nullptr);
}

// resident blocks of 128 threads per SM the register budget is sized for (a
// tuning knob of the build: 3 caps a thread at 168 registers, 2 at 255)
#ifndef BATCH_BLOCKS_128
#define BATCH_BLOCKS_128 3
#endif

// UNI != UNI_NONE: every instance has the launch's model and cost (a.model, a.cost)
template <int BLOCK, int UNI>
__global__ void __launch_bounds__(BLOCK, BLOCK == 256 ? 1 : (BLOCK == 128 ? BATCH_BLOCKS_128 : 384 / BLOCK))
    k_batch(const __grid_constant__ BatchArgs a) {
    __shared__ InstDesc sd;
    __shared__ int s_item, s_last;
    trig_to_shared();
    const int tid = threadIdx.x, leg = tid & 3, r = tid >> 2;
    const int n_items = *a.n_items;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        {
            const int* src = reinterpret_cast<const int*>(a.desc + w.inst);
            int* dst = reinterpret_cast<int*>(&sd);
            for (int i = tid; i < (int)(sizeof(InstDesc) / 4); i += BLOCK) dst[i] = __ldcg(src + i);
        }
        __syncthreads();
        const bool valid = r < w.n;
        const int k = w.k0 + (valid ? r : w.n - 1);
        const uint32_t step = __ldcg(a.steps + w.inst);
        float Uk[NKNOT][3];
        sample_lane(sd, k, leg, step, valid, Uk);
        // gait time of this horizon: step * control period, reduced modulo the gait period
        const double t0d = (double)step * sd.ctrl_steps * sd.dt_d;
        const float t0 = ((sd.gait == 1 || sd.gait == 2) && sd.period_d > 0) ? (float)fmod(t0d, sd.period_d)
                                                                          : (float)t0d;
        const HorizonArgs hz = {sd.H, sd.n_sub, sd.nx, sd.h, sd.dt, sd.inv_Hm1, t0, sd.arm, sd.interp, sd.Bt};
        const float* x0 = a.x0s + (size_t)w.inst * NX_BOX;
        const float L = UNI != UNI_NONE ? rollout_item<UNI>(a.model, a.cost, hz, x0, Uk, leg, k, valid)
                                        : rollout_item<UNI>(sd.model, sd.cost, hz, x0, Uk, leg, k, valid);
        if (valid && leg == 0) sd.L[k] = L;
        if (cta_count_in(a.done + w.inst, (unsigned)w.n, (unsigned)sd.K, s_last)) {
            block_update<BLOCK>(sd, a.u0s + (size_t)w.inst * NJ);
            if (tid == 0) a.done[w.inst] = 0u;
        }
        __syncthreads();
    }
}

template <int BLOCK, int UNI>
cudaError_t launch_k_batch(const BatchArgs& a, int grid, cudaStream_t st) {
    k_batch<BLOCK, UNI><<<grid, BLOCK, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
