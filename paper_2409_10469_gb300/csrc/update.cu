// update.cu -- K3/K4: softmax weights (Eq. 1), weighted mean (Eq. 2), applied
// control u = mu[0] and the receding-horizon shift (Alg. 1, last steps) of
// arXiv 2409.10469, Sec. II-B.
//
// G CTAs split the n samples into contiguous chunks of about 128 (a second grid
// dimension T tiles the 12 H parameters of direct targets into groups of 48;
// the knot representations have one tile and their own kernel).  Every CTA
// reads only its chunk's costs: their minimum m_c over the finite ones, the
// weights w_k = exp(-(L_k - m_c)/lambda) (0 if L_k is not finite) with the
// exponent and the exp in FP64, computed once per sample into shared memory as
// FP32 pairs (about 48 significant bits), their sum z_c and the sums
// S_c = sum_k w_k U_k of its tile's parameters (float-float pairs per lane,
// across lanes and warps: FP64 runs at 1/64 of the FP32 rate on this part, so
// beyond the exps only the last CTA's combine uses it).  It writes these and m_c
// to scratch and bumps a counter; the CTA that sees the counter reach the grid
// size - 1 (no waiting: it is simply the last to finish) takes L_min = min_c m_c
// and scales chunk c by f_c = exp(-(m_c - L_min)/lambda) (FP64) -- Eq. 1's
// weights factor as exp(-(L_k - L_min)/lambda) = w_k f_c -- so that
// mu' = sum_c f_c S_c / sum_c f_c z_c.  The chunks are added in a fixed order and
// tree, so the result does not depend on scheduling.  It writes mu', u0 = the
// controls of step 0 (knot 0, or the first direct target), the shifted nominal
// and the status, and re-arms the counter for the next launch.
#include "kernels.h"

namespace mppi {

constexpr int UPD_THREADS = 256;
constexpr int UPD_WARPS = UPD_THREADS / 32;
constexpr int UPD_TILE = D;   // parameters per dimension tile

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= 3.402823466e38f; }

// float-float accumulation: (s, e) += (v, ve), s + v split exactly into the new
// s and an error term by Knuth's TwoSum, the error and the low parts into e
// (about 48 significant bits on the FP32 pipe, which runs 64x the FP64 rate)
__device__ __forceinline__ void ff_acc(float& s, float& e, float v, float ve) {
    // _rn intrinsics: never contracted with a preceding product (which would break TwoSum)
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    e = __fadd_rn(e, __fadd_rn(ve, err));
}

constexpr int UPD_SUB = UPD_THREADS;  // samples whose weights sit in shared memory at a time

// One warp's share of a sub-chunk: samples k = kb, kb + UPD_WARPS, ... < ke, the
// lane's parameter pair u2[k * row2] times the weight pair w[k - ks] (the
// products' rounding errors by FMA) into float-float sums (s, e), one sample at
// a time in order; the loads of 8 samples are issued together (one L2 round
// trip each)
__device__ __forceinline__ void sum_chunk(const float2* w, int ks, const float2* u2, int row2, int kb, int ke,
                                          float& s0, float& s1, float& e0, float& e1) {
    constexpr int NB = 8;
    for (int kk = kb; kk < ke; kk += NB * UPD_WARPS) {
        float2 ub[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int k = kk + q * UPD_WARPS;
            ub[q] = k < ke ? __ldg(u2 + (size_t)k * row2) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int k = kk + q * UPD_WARPS;
            if (k >= ke) break;
            const float2 wk = w[k - ks];
            const float2 u = ub[q];
            const float p0 = wk.x * u.x, p1 = wk.x * u.y;
            ff_acc(s0, e0, p0, fmaf(wk.y, u.x, fmaf(wk.x, u.x, -p0)));
            ff_acc(s1, e1, p1, fmaf(wk.y, u.y, fmaf(wk.x, u.y, -p1)));
        }
    }
}

constexpr int UPD_NB = 8;             // chunk partials a combining lane loads per round trip
constexpr int UPD_ROW = UPD_TILE + 2;  // a chunk's scratch row: 48 sums, z_c, m_c
static_assert(UPDATE_MAX_CTAS <= UPD_THREADS, "the last CTA holds one chunk per thread");

struct UpdSmem {
    float red[UPD_WARPS];
    float2 z[UPD_WARPS];              // per-warp weight sums (hi, lo)
    float2 part[UPD_WARPS][UPD_TILE];  // per-warp parameter sums (hi, lo)
    float2 w[UPD_SUB];                 // a sub-chunk's weights (hi, lo)
    double f[UPDATE_MAX_CTAS];  // the chunks' factors exp(-(m_c - L_min) / lambda)
    double Z;
    float Lmin;  // the minimum over the chunks' cost minima (combine_setup)
    int last;
};

// minimum of v over the CTA, returned to every thread
__device__ __forceinline__ float block_min(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();  // red is free
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int w = 1; w < UPD_WARPS; w++) m = fminf(m, red[w]);
    return m;
}

// CTA b's chunk on the parameter tile starting at d0: its row of the tile's
// scratch gets S_c of the tile's parameters, then z_c and m_c.  With PRE the
// chunk's weights, z_c and m_c come from k_update_weights (a.wts, a.zm) instead
// of being formed here (direct targets: every tile would repeat the FP64 exps).
template <bool PRE>
__device__ __forceinline__ void chunk_partials(const UpdateArgs& a, int b, int G, int d0, double* rows, UpdSmem& s) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Dp = a.Dp;
    const int chunk = (a.n + G - 1) / G;
    const int k0 = b * chunk, k1 = min(a.n, k0 + chunk);
    float m;
    if (PRE) {
        m = (float)__ldcg(a.zm + 2 * b + 1);
    } else {
        float lm = INFINITY;
        for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
            const float l = __ldg(a.L + k);
            if (finitef(l)) lm = fminf(lm, l);
        }
        m = block_min(lm, s.red);
    }
    const bool okc = finitef(m);
    // sum_k w_k U_k: warp w takes samples ks + w, ks + w + 8, ... of each
    // sub-chunk; lane i < 24 owns parameters d0 + 2i, d0 + 2i + 1 (Dp is even, so
    // a pair never straddles the end)
    const bool own = lane < UPD_TILE / 2 && d0 + 2 * lane < Dp;
    const float2* u2 = reinterpret_cast<const float2*>(a.U + d0) + lane;
    float zs = 0.f, ze = 0.f;
    float s0 = 0.f, s1 = 0.f, e0 = 0.f, e1 = 0.f;
    if (okc)
        for (int ks = k0; ks < k1; ks += UPD_SUB) {
            // Eq. 1's weights around the chunk minimum, once per sample: exponent
            // and exp in FP64, kept as pairs
            const int k = ks + tid;
            float2 wk = make_float2(0.f, 0.f);
            if (PRE) {
                if (k < k1) wk = __ldcg(a.wts + k);
            } else if (k < k1) {
                const float l = __ldg(a.L + k);
                if (finitef(l)) {
                    const double wd = exp(-((double)l - (double)m) * a.inv_lambda);
                    wk.x = (float)wd;
                    wk.y = (float)(wd - (double)wk.x);
                }
            }
            if (!PRE) ff_acc(zs, ze, wk.x, wk.y);
            __syncthreads();  // the previous sub-chunk's weights are consumed
            s.w[tid] = wk;
            __syncthreads();
            if (own) sum_chunk(s.w, ks, u2, Dp / 2, ks + warp, min(k1, ks + UPD_SUB), s0, s1, e0, e1);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, zs, o), ve = __shfl_xor_sync(0xffffffffu, ze, o);
        ff_acc(zs, ze, v, ve);
    }
    if (lane == 0) s.z[warp] = make_float2(zs, ze);
    if (lane < UPD_TILE / 2) {
        s.part[warp][2 * lane] = make_float2(s0, e0);
        s.part[warp][2 * lane + 1] = make_float2(s1, e1);
    }
    __syncthreads();
    // the warps' pairs added in warp order; the row holds hi + lo as a double
    double* row = rows + (size_t)b * UPD_ROW;
    if (tid < UPD_TILE && d0 + tid < Dp) {
        float hi = s.part[0][tid].x, lo = s.part[0][tid].y;
        for (int w = 1; w < UPD_WARPS; w++) ff_acc(hi, lo, s.part[w][tid].x, s.part[w][tid].y);
        row[tid] = (double)hi + (double)lo;
    }
    if (tid == UPD_TILE) {
        if (PRE) {
            row[UPD_TILE] = __ldcg(a.zm + 2 * b);
        } else {
            float hi = s.z[0].x, lo = s.z[0].y;
            for (int w = 1; w < UPD_WARPS; w++) ff_acc(hi, lo, s.z[w].x, s.z[w].y);
            row[UPD_TILE] = (double)hi + (double)lo;
        }
    }
    if (tid == UPD_TILE + 1) row[UPD_TILE + 1] = (double)m;
}

// Direct targets, first pass: chunk b's cost minimum m_c, its samples' weights
// exp(-(L_k - m_c) / lambda) (exponent and exp in FP64, kept as FP32 pairs) into
// a.wts and z_c = their sum into a.zm -- once per sample, for every parameter
// tile of the second pass
__global__ void __launch_bounds__(UPD_THREADS) k_update_weights(UpdateArgs a) {
    __shared__ float red[UPD_WARPS];
    __shared__ float2 zw[UPD_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, b = blockIdx.x, G = gridDim.x;
    const int chunk = (a.n + G - 1) / G;
    const int k0 = b * chunk, k1 = min(a.n, k0 + chunk);
    float lm = INFINITY;
    for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
        const float l = __ldg(a.L + k);
        if (finitef(l)) lm = fminf(lm, l);
    }
    const float m = block_min(lm, red);
    const bool okc = finitef(m);
    float zs = 0.f, ze = 0.f;
    for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
        const float l = __ldg(a.L + k);
        float2 wk = make_float2(0.f, 0.f);
        if (okc && finitef(l)) {
            const double wd = exp(-((double)l - (double)m) * a.inv_lambda);
            wk.x = (float)wd;
            wk.y = (float)(wd - (double)wk.x);
        }
        a.wts[k] = wk;
        ff_acc(zs, ze, wk.x, wk.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, zs, o), ve = __shfl_xor_sync(0xffffffffu, ze, o);
        ff_acc(zs, ze, v, ve);
    }
    if (lane == 0) zw[warp] = make_float2(zs, ze);
    __syncthreads();
    if (tid == 0) {
        float hi = zw[0].x, lo = zw[0].y;
        for (int w = 1; w < UPD_WARPS; w++) ff_acc(hi, lo, zw[w].x, zw[w].y);
        a.zm[2 * b] = (double)hi + (double)lo;
        a.zm[2 * b + 1] = (double)m;
    }
}

// publish this CTA's writes and count it in: true in the last of `total` CTAs
__device__ __forceinline__ bool count_in(unsigned* counter, unsigned total, UpdSmem& s) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s.last = (atomicAdd(counter, 1u) == total - 1);
    __syncthreads();
    if (!s.last) return false;
    __threadfence();
    return true;
}

// the last CTA of a tile: L_min over the G chunk minima of the tile's rows, the
// factors f_c, and Z = sum_c f_c z_c (warp 0: lane j takes chunks j, j + 32, ...
// in order, then a fixed xor tree).  Returns whether any cost is finite.
__device__ __forceinline__ bool combine_setup(const UpdateArgs& a, int G, const double* rows, UpdSmem& s) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float mc = tid < G ? (float)__ldcg(rows + (size_t)tid * UPD_ROW + UPD_TILE + 1) : INFINITY;
    const float Lmin = block_min(mc, s.red);
    const bool ok = finitef(Lmin);
    if (tid == 0) s.Lmin = Lmin;
    if (tid < G) s.f[tid] = (ok && finitef(mc)) ? exp(-((double)mc - (double)Lmin) * a.inv_lambda) : 0.0;
    __syncthreads();
    if (warp == 0) {
        constexpr int NQ = UPDATE_MAX_CTAS / 32;
        double v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int c = lane + 32 * q;
            v[q] = c < G ? __ldcg(rows + (size_t)c * UPD_ROW + UPD_TILE) : 0.0;
        }
        double z = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int c = lane + 32 * q;
            if (c < G) z = fma(s.f[c], v[q], z);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (lane == 0) s.Z = z;
    }
    __syncthreads();
    return ok;
}

// S_j = sum_c f_c S_c[j] for tile parameter j by the 4 lanes q of a quad (chunks
// c = q mod 4 in order, UPD_NB loads per round trip), added over the quad by a
// fixed xor tree; every lane of the quad returns it.  The whole warp calls it.
__device__ __forceinline__ double combine_param(int G, const double* rows, int j, int q, const UpdSmem& s) {
    double acc = 0.0;
    for (int c0 = q; c0 < G; c0 += 4 * UPD_NB) {
        double v[UPD_NB];
#pragma unroll
        for (int i = 0; i < UPD_NB; i++) {
            const int c = c0 + 4 * i;
            v[i] = c < G ? __ldcg(rows + (size_t)c * UPD_ROW + j) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < UPD_NB; i++) {
            const int c = c0 + 4 * i;
            if (c < G) acc = fma(s.f[c], v[i], acc);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    return acc;
}

// Knot representations (48 parameters): one parameter tile.
__global__ void __launch_bounds__(UPD_THREADS) k_update_knots(UpdateArgs a) {
    __shared__ UpdSmem s;
    __shared__ float s_mu[D];
    const int tid = threadIdx.x, G = gridDim.x;
    chunk_partials<false>(a, blockIdx.x, G, 0, a.part, s);
    if (!count_in(a.counter, (unsigned)G, s)) return;

    // last CTA: combine, apply, shift
    const bool ok = combine_setup(a, G, a.part, s);
    {
        const int j = tid >> 2, q = tid & 3;  // 64 quads, 48 parameters
        const double S = combine_param(G, a.part, min(j, D - 1), q, s);
        if (j < D && q == 0) {
            // every cost non-finite: keep the previous mean
            const float mu_new = ok ? (float)(S / s.Z) : a.mu[j];
            s_mu[j] = mu_new;
            if (a.mu_upd) a.mu_upd[j] = mu_new;
            if (j < NJ) a.u0[j] = mu_new;  // the spline at tau = 0 is knot 0
        }
    }
    if (tid == 0) {
        if (ok && a.wsum) *a.wsum = s.Z;
        if (a.status) *a.status = ok ? 0 : 4;
        *a.counter = 0u;  // re-arm for the next launch (kernels on one stream are ordered)
    }
    __syncthreads();
    // shifted(mu): the representation's interpolant re-sampled at tau_j + delta,
    // held at tau = 1 past the end
    if (tid < D) a.mu[tid] = shifted_knot(s_mu, a.interp, a.H, a.ctrl_steps, tid / NJ, tid % NJ);
}

// The partial sums of a shard of a K-sample step (knot representations): the
// chunks as in k_update_knots, then the last CTA writes the shard's minimum
// m = min_c m_c, Z = sum_c f_c z_c and S_j = sum_c f_c S_c[j] (f_c relative to m)
// to partial_out instead of dividing and shifting.  Every rank of a sharded
// step rescales these by exp(-(m - L_min) / lambda) once the global L_min is
// known; the sums over ranks are Eq. 2's numerator and denominator.
__global__ void __launch_bounds__(UPD_THREADS) k_update_partial(UpdateArgs a) {
    __shared__ UpdSmem s;
    const int tid = threadIdx.x, G = gridDim.x;
    chunk_partials<false>(a, blockIdx.x, G, 0, a.part, s);
    if (!count_in(a.counter, (unsigned)G, s)) return;
    const bool ok = combine_setup(a, G, a.part, s);
    {
        const int j = tid >> 2, q = tid & 3;
        const double S = combine_param(G, a.part, min(j, D - 1), q, s);
        if (j < D && q == 0) a.partial_out[2 + j] = ok ? S : 0.0;
    }
    if (tid == 0) {
        a.partial_out[0] = (double)s.Lmin;
        a.partial_out[1] = ok ? s.Z : 0.0;
        *a.counter = 0u;  // re-arm for the next launch
    }
}

// mu' = S / Z from the sums of every shard, u0, the status and the shift (one CTA)
__global__ void k_update_finalize(FinalizeArgs a) {
    __shared__ float s_mu[D];
    const int tid = threadIdx.x;
    const double Z = a.sums[0];
    const bool ok = Z > 0.0 && Z <= 1.79769313486231570e308;
    for (int j = tid; j < D; j += blockDim.x) {
        const float mu_new = ok ? (float)(a.sums[1 + j] / Z) : a.mu[j];  // no finite cost: keep the mean
        s_mu[j] = mu_new;
        a.mu_upd[j] = mu_new;
        if (j < NJ) a.u0[j] = mu_new;
    }
    if (tid == 0) *a.status = ok ? 0 : 4;
    __syncthreads();
    for (int j = tid; j < D; j += blockDim.x) a.mu[j] = shifted_knot(s_mu, a.interp, a.H, a.ctrl_steps, j / NJ, j % NJ);
}

// Direct targets (12 H parameters): G x T CTAs, T = ceil(12 H / 48) parameter
// tiles, each tile its own update: the last CTA of tile y (counter[1 + y])
// combines the tile's 48 parameters from its G rows (every tile's rows carry
// z_c and m_c, computed identically); the last tile to finish (counter[0])
// applies the shift, which moves targets across tiles.
__global__ void __launch_bounds__(UPD_THREADS) k_update_tiled(UpdateArgs a) {
    __shared__ UpdSmem s;
    const int tid = threadIdx.x, G = gridDim.x, T = gridDim.y, y = blockIdx.y;
    const int Dp = a.Dp, d0 = y * UPD_TILE;
    double* rows = a.part + (size_t)y * G * UPD_ROW;
    chunk_partials<true>(a, blockIdx.x, G, d0, rows, s);
    if (!count_in(a.counter + 1 + y, (unsigned)G, s)) return;

    // last CTA of this tile: combine and apply its parameters
    const bool ok = combine_setup(a, G, rows, s);
    {
        const int j = tid >> 2, q = tid & 3, d = d0 + j;
        const double S = combine_param(G, rows, min(j, UPD_TILE - 1), q, s);
        if (j < UPD_TILE && d < Dp && q == 0) {
            const float mu_new = ok ? (float)(S / s.Z) : a.mu[d];  // every cost non-finite: keep the mean
            a.mu_upd[d] = mu_new;
            if (d < NJ) a.u0[d] = mu_new;  // the controls of step 0: the first direct target
        }
    }
    if (tid == 0) {
        if (y == 0) {
            if (ok && a.wsum) *a.wsum = s.Z;
            if (a.status) *a.status = ok ? 0 : 4;
        }
        a.counter[1 + y] = 0u;  // re-arm for the next launch
    }
    if (!count_in(a.counter, (unsigned)T, s)) return;
    // the last tile: direct targets move ctrl_steps steps earlier, the last one
    // held (every tile's mu_upd was published before its count)
    for (int d = tid; d < Dp; d += UPD_THREADS) {
        const int t = d / NJ, i = d % NJ;
        const int src = min(t + a.ctrl_steps, a.H - 1);
        a.mu[d] = __ldcg(a.mu_upd + src * NJ + i);
    }
    if (tid == 0) a.counter[0] = 0u;
}

int update_grid(int n) {
    int g = (n + 127) / 128;  // ~128 samples per CTA (measured: 64 per CTA costs 3 us more at n = 4096)
    return g < 1 ? 1 : (g > UPDATE_MAX_CTAS ? UPDATE_MAX_CTAS : g);
}

// direct targets: chunks of ~128 samples (x T parameter tiles), as the knots
static int update_grid_tiled(int n) {
    int g = (n + 127) / 128;
    return g < 1 ? 1 : (g > UPDATE_MAX_CTAS ? UPDATE_MAX_CTAS : g);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
    if (a.Dp % 2 != 0 || a.Dp < D || (a.Dp > D && !a.mu_upd)) return cudaErrorInvalidValue;
    if (a.Dp == D) {
        k_update_knots<<<update_grid(a.n), UPD_THREADS, 0, st>>>(a);
    } else {
        if (!a.wts || !a.zm) return cudaErrorInvalidValue;
        k_update_weights<<<update_grid_tiled(a.n), UPD_THREADS, 0, st>>>(a);
        const dim3 grid(update_grid_tiled(a.n), (a.Dp + UPD_TILE - 1) / UPD_TILE);
        k_update_tiled<<<grid, UPD_THREADS, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_update_partial(const UpdateArgs& a, cudaStream_t st) {
    if (a.Dp != D || !a.partial_out) return cudaErrorInvalidValue;
    k_update_partial<<<update_grid(a.n), UPD_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update_finalize(const FinalizeArgs& a, cudaStream_t st) {
    k_update_finalize<<<1, 64, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
