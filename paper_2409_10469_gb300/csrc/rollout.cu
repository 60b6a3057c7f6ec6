// rollout.cu -- K2: MPPI rollouts of one instance on sm_103a CUDA cores (FP32).
//
// arXiv 2409.10469, Alg. 1 inner loop: every sample's knot vector is turned into
// joint targets by the cubic spline (Sec. III-B), tracked by PD (Sec. IV-A) and
// simulated for T steps while L_walk (Sec. IV-B) and L_box (Sec. IV-D) accumulate.
// The per-lane arithmetic lives in rollout.cuh; this kernel maps 4 lanes to a
// rollout (8 rollouts per warp) over the n samples of one controller.  In the
// control step it also samples the knots (Alg. 1's sampling) and ends with the
// update (Eq. 1, Eq. 2, apply, shift), so a step is one launch.
#include "kernels.h"
#include "noise.cuh"
#include "rollout.cuh"

namespace mppi {

__device__ __forceinline__ bool fin_f(float x) { return fabsf(x) <= 3.402823466e38f; }

// The update of the control step fused into the rollout kernel (knot
// representations).  Eq. 1 weights exp(-(L_k - L_min) / lambda) factor as
// exp(-(L_k - m_c) / lambda) exp(-(m_c - L_min) / lambda) for any m_c, so each CTA
// takes m_c = the minimum of its own finite costs and weights its rollouts by the
// first factor.  Both factors -- the exponent (L - m) / lambda and its exp -- are
// formed in FP64 (one exp per rollout and one per CTA: a few microseconds of the
// FP64 pipe, which runs at 1/64 of the FP32 rate on this part) and split into an
// FP32 pair (hi, lo) that carries about 48 significant bits.  The sums of w and
// w U are compensated FP32 pairs (hi, lo) -- Knuth's TwoSum for additions, an
// FMA for the rounding error of products -- at the FP32 rate: over the warp's 8
// rollouts (lanes of the same leg), then over the warps in order.  The CTA writes
// (sums, m_c) and counts itself in; the last CTA (every other CTA has finished,
// so none still reads the nominal) takes L_min = min m_c and the factors
// f_c = exp(-(m_c - L_min) / lambda), and for each of the 49 sums groups of
// threads add f_c times the CTA partials over contiguous ranges of c, in four
// interleaved accumulators each, all combined in a fixed order (32 partials
// loaded per round trip); mu' = S / Z (a float-float quotient), u0, the status and the
// shifted nominal follow, and the counter is re-armed.  Every thread of the CTA
// calls this (it synchronises the block).

// (s, e) += (v, ve): s + v exactly as s' + err (Knuth's TwoSum), err and the low
// parts into e
__device__ __forceinline__ void ff_add(float& s, float& e, float v, float ve) {
    // _rn intrinsics: never contracted with a preceding product (which would break TwoSum)
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    e = __fadd_rn(e, __fadd_rn(ve, err));
}

__device__ __forceinline__ void fused_update(const RolloutArgs& a, float L, const float (&Uk)[NKNOT][3], int leg,
                                             bool valid) {
    __shared__ float s_m[8];
    __shared__ float2 s_sum[8][FUSE_W];
    __shared__ float2 s_f[FUSE_MAX_CTAS];
    __shared__ float s_mu[D];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, B = blockDim.x;
    const int G = gridDim.x;
    float2* part = reinterpret_cast<float2*>(a.part);  // [G][FUSE_W] (hi, lo); entry D + 1 holds (m_c, 0)
    // this CTA's minimum finite cost
    const bool fin = valid && fin_f(L);
    float m = fin ? L : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_m[warp] = m;
    __syncthreads();
    float mc = s_m[0];
    for (int w = 1; w < nw; w++) mc = fminf(mc, s_m[w]);
    // Eq. 1's weight around the CTA minimum: exponent and exp in FP64, kept as
    // the pair wh + wl
    const double wk = (fin && fin_f(mc)) ? exp(-((double)L - (double)mc) * a.inv_lambda) : 0.0;
    const float wh = (float)wk, wl = (float)(wk - (double)wh);
    // products w U_k with their rounding errors and the weight's low part
    float hs[NKNOT][3], he[NKNOT][3];
#pragma unroll
    for (int j = 0; j < NKNOT; j++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            hs[j][i] = wh * Uk[j][i];
            he[j][i] = fmaf(wl, Uk[j][i], fmaf(wh, Uk[j][i], -hs[j][i]));
        }
    float zs = leg == 0 ? wh : 0.f, ze = leg == 0 ? wl : 0.f;  // one weight per rollout
    // the warp's 8 rollouts: lanes leg, leg + 4, ..., leg + 28
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        {
            const float v = __shfl_xor_sync(0xffffffffu, zs, o), ve = __shfl_xor_sync(0xffffffffu, ze, o);
            ff_add(zs, ze, v, ve);
        }
#pragma unroll
        for (int j = 0; j < NKNOT; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float v = __shfl_xor_sync(0xffffffffu, hs[j][i], o);
                const float ve = __shfl_xor_sync(0xffffffffu, he[j][i], o);
                ff_add(hs[j][i], he[j][i], v, ve);
            }
    }
    if (lane < 4) {
#pragma unroll
        for (int j = 0; j < NKNOT; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) s_sum[warp][j * NJ + 3 * lane + i] = make_float2(hs[j][i], he[j][i]);
        if (lane == 0) s_sum[warp][D] = make_float2(zs, ze);
    }
    __syncthreads();
    float2* mine = part + (size_t)blockIdx.x * FUSE_W;
    for (int d = tid; d <= D; d += B) {
        float hi = s_sum[0][d].x, lo = s_sum[0][d].y;
        for (int w = 1; w < nw; w++) ff_add(hi, lo, s_sum[w][d].x, s_sum[w][d].y);
        mine[d] = make_float2(hi, lo);
    }
    if (tid == 0) mine[D + 1] = make_float2(mc, 0.f);
    // publish, then count this CTA in
    if (!cta_count_in(a.counter, 1u, (unsigned)G, s_last)) return;

    // ---- last CTA: L_min over the CTA minima (kept in s_f for the factors)
    float M = INFINITY;
    for (int c = tid; c < G; c += B) {
        const float mcc = __ldcg(part + (size_t)c * FUSE_W + D + 1).x;
        s_f[c].x = mcc;
        M = fminf(M, mcc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M = fminf(M, __shfl_xor_sync(0xffffffffu, M, o));
    __syncthreads();
    if (lane == 0) s_m[warp] = M;
    __syncthreads();
    M = s_m[0];
    for (int w = 1; w < nw; w++) M = fminf(M, s_m[w]);
    const bool ok = fin_f(M);
    // the factors exp(-(m_c - L_min) / lambda) in FP64, kept as pairs (0 for a CTA
    // without a finite cost)
    for (int c = tid; c < G; c += B) {
        const float mcc = s_f[c].x;
        const double f = (ok && fin_f(mcc)) ? exp(-((double)mcc - (double)M) * a.inv_lambda) : 0.0;
        const float fh = (float)f;
        s_f[c] = make_float2(fh, (float)(f - (double)fh));
    }
    __syncthreads();
    // each of the 49 sums over the CTAs: thread group g (64 threads, one per sum)
    // takes a contiguous range of CTAs, in four accumulators (the range's c mod 4)
    // fed 32 partials per round trip; accumulators and groups are combined in order
    constexpr int BATCH = 32;
    const int ng = B >= 64 ? B / 64 : 1, dstep = B >= 64 ? 64 : B, g = B >= 64 ? tid / 64 : 0;
    const int crange = (G + ng - 1) / ng, cb = g * crange, ce = min(G, cb + crange);
    for (int d = B >= 64 ? tid % 64 : tid; d <= D; d += dstep) {
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        if (ok) {
            const float2* pd = part + d;
            for (int c = cb; c < ce; c += BATCH) {
                float2 v[BATCH];
#pragma unroll
                for (int q = 0; q < BATCH; q++)
                    v[q] = c + q < ce ? __ldcg(pd + (size_t)(c + q) * FUSE_W) : make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < BATCH; q++) {
                    const float2 f = c + q < ce ? s_f[c + q] : make_float2(0.f, 0.f);
                    const float p = f.x * v[q].x;
                    ff_add(hi[q & 3], lo[q & 3], p, fmaf(f.y, v[q].x, fmaf(f.x, v[q].y, fmaf(f.x, v[q].x, -p))));
                }
            }
        }
#pragma unroll
        for (int q = 1; q < 4; q++) ff_add(hi[0], lo[0], hi[q], lo[q]);
        s_sum[g][d] = make_float2(hi[0], lo[0]);
    }
    __syncthreads();
    for (int d = tid; d <= D; d += B) {
        float hi = s_sum[0][d].x, lo = s_sum[0][d].y;
        for (int gg = 1; gg < ng; gg++) ff_add(hi, lo, s_sum[gg][d].x, s_sum[gg][d].y);
        s_sum[0][d] = make_float2(hi, lo);
    }
    __syncthreads();
    for (int d = tid; d < D; d += B) {
        // no finite cost: keep the mean; the quotient of the pairs on the FP32 pipe
        const float mu_new = ok ? ff_div(s_sum[0][d], s_sum[0][D]) : a.mu_w[d];
        s_mu[d] = mu_new;
        if (a.mu_upd) a.mu_upd[d] = mu_new;
        if (a.mu_host) a.mu_host[d] = mu_new;
        if (d < NJ) {
            a.u0[d] = mu_new;  // the spline at tau = 0 is knot 0
            if (a.u0_host) a.u0_host[d] = mu_new;
        }
    }
    if (tid == 0) {
        if (a.wsum && ok) *a.wsum = (double)s_sum[0][D].x + (double)s_sum[0][D].y;
        if (a.status) *a.status = ok ? 0 : 4;
        if (a.status_host) *a.status_host = ok ? 0 : 4;
        *a.counter = 0u;  // re-arm for the next launch (kernels on one stream are ordered)
    }
    __syncthreads();
    // shifted(mu'): the representation's interpolant re-sampled at tau_j + delta
    for (int d = tid; d < D; d += B) a.mu_w[d] = shifted_knot(s_mu, a.interp, a.H, a.ctrl_steps, d / NJ, d % NJ);
}

template <int TERR, bool BOX, bool DIRECT>
__global__ void __launch_bounds__(256, 1) k_rollout(RolloutArgs a) {
    trig_to_shared();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt >> 2, leg = gt & 3;
    const bool valid = k < a.n;
    const int kk = valid ? k : a.n - 1;
    const int nx = a.model.nx;
    const float* x0 = a.x0 + (a.x0_per_sample ? (size_t)kk * nx : 0);
    float Uk[NKNOT][3];
    const float* Urow = a.U + (size_t)kk * a.Dp;
    if (!DIRECT && a.sample) {
        // Alg. 1's sampling step for this lane's knots, element for element the
        // formula of k_sample (Philox counter (d / 4, k, step, inst), Box-Muller,
        // fmaf perturbation, clamp), so the knots are bit-identical to it; kg is
        // the sample's index in the whole K-sample step (a shard starts at k_off)
        const int kg = a.k_off + kk;
        const int kp0 = a.K_all - (a.mu_prop ? a.n_prop : 0);
        const bool prop = a.mu_prop && kg >= kp0;
        const float* ctr = prop ? a.mu_prop : a.mu;
        const bool nominal = (kg == 0) || (prop && kg == kp0);
#pragma unroll
        for (int j = 0; j < NKNOT; j++) {
            const int d0 = j * NJ + 3 * leg;
            float epsv[3];
            knot_normals(a.key0, a.key1, a.step, a.inst, (uint32_t)kg, d0, epsv);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int d = d0 + i;
                const float eps = nominal ? 0.f : epsv[i];
                float c = __ldg(ctr + d);
                if (prop && !(fabsf(c) <= 3.402823466e38f)) c = __ldg(a.mu + d);  // non-finite proposal: plain mean
                const float v = fminf(fmaxf(__fmaf_rn(a.sigma[d], eps, c), a.q_lo[i]), a.q_hi[i]);
                Uk[j][i] = v;
                if (valid) a.U_out[(size_t)kk * D + d] = v;
            }
        }
    } else if (!DIRECT) {
#pragma unroll
        for (int j = 0; j < NKNOT; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) Uk[j][i] = Urow[j * NJ + 3 * leg + i];
    } else {
#pragma unroll
        for (int j = 0; j < NKNOT; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) Uk[j][i] = 0.f;
    }
    const HorizonArgs hz = {a.H, a.n_sub, nx, a.h, a.dt, a.inv_Hm1, a.t0, a.arm, a.interp, a.Bt};
    const float L = rollout_lane<TERR, BOX, DIRECT>(a.model, a.cost, hz, x0, Uk, Urow, leg, k, valid, a.traj);
    if (valid && leg == 0) a.L[k] = L;
    if (!DIRECT && a.fuse) fused_update(a, L, Uk, leg, valid);
}

template <int TERR, bool BOX>
static cudaError_t launch_t(const RolloutArgs& a, int block, cudaStream_t st) {
    long threads = 4L * a.n;
    int grid = (int)((threads + block - 1) / block);
    if (a.interp == INTERP_DIRECT) k_rollout<TERR, BOX, true><<<grid, block, 0, st>>>(a);
    else k_rollout<TERR, BOX, false><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rollout(const RolloutArgs& a, int block, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const bool box = a.model.has_box != 0;
    // 0: flat plane and no static boxes (specialised); 1: plane or heightfield with static boxes
    if (a.model.terrain != 0 || a.model.n_sbox > 0)
        return box ? launch_t<1, true>(a, block, st) : launch_t<1, false>(a, block, st);
    return box ? launch_t<0, true>(a, block, st) : launch_t<0, false>(a, block, st);
}

}  // namespace mppi
