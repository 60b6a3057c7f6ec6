// update.cu -- K3/K4: softmax weights (Eq. 1), weighted mean (Eq. 2), applied
// control u = mu[0] and the receding-horizon shift (Alg. 1, last steps) of
// arXiv 2409.10469, Sec. II-B.
//
// Knot representations (48 parameters): G CTAs split the n samples into
// contiguous chunks of about 128.  Every CTA reads only its chunk's costs: their
// minimum m_c over the finite ones, the weights w_k = exp(-(L_k - m_c)/lambda)
// (0 if L_k is not finite) with the exponent and the exp in FP64, computed once
// per sample into shared memory as FP32 pairs (about 48 significant bits), their
// sum z_c and the sums S_c = sum_k w_k U_k (float-float pairs per lane, across
// lanes and warps: FP64 runs at 1/64 of the FP32 rate on this part, so only the
// exps use it).  It writes these pairs and m_c to scratch and bumps a counter;
// the CTA that sees the counter reach the grid size - 1 (no waiting: it is
// simply the last to finish) takes L_min = min_c m_c and scales chunk c by
// f_c = exp(-(m_c - L_min)/lambda) (FP64, kept as a pair) -- Eq. 1's weights
// factor as exp(-(L_k - L_min)/lambda) = w_k f_c -- so that
// mu' = sum_c f_c S_c / sum_c f_c z_c, the sums and the quotient in float-float.
// The chunks are added in a fixed order and tree, so the result does not depend
// on scheduling.  It writes mu', u0 = the controls of step 0 (knot 0), the
// shifted nominal and the status, and re-arms the counter for the next launch.
//
// Direct targets (12 H parameters per sample, rows of kilobytes) take Eq. 1's
// weights around the global minimum directly, in three launches: k_update_lmin
// finds L_min over the finite costs (an atomic max on an order-reversed integer
// key, so the result does not depend on scheduling); k_update_rows streams U
// row by row -- CTA (c, y), two per SM, takes chunk c of the samples and column
// tile y of the parameters, each thread one 16-byte group of every row, so a
// warp reads 512 contiguous bytes per row -- with the weights
// w_k = exp(-(L_k - L_min)/lambda) (FP64 exponent and exp); it adds the rows two
// at a time in FP32, w_a u_a + w_b u_b by one product and one FMA, into
// float-float sums, and writes its chunk's sums of its tile and, from tile 0,
// z_c = sum w_k (float-float from the FP64 weights); k_update_combine adds the
// chunks per column in float-float by a fixed tree (no factors: every chunk
// shares the reference L_min) and its last CTA shifts.  Error of the two-row
// FP32 step: at most 3 roundings of 2^-24 (the product, the FMA, the weight's
// FP32 rounding) of sum_k w_k |u_kj|, so |mu'_j error| <= 1.8e-7 max_k |u_kj|.
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
constexpr int UPD_PF = 16;            // a warp's samples whose loads go out before the weights are known

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
    float2 f[UPDATE_MAX_CTAS];  // the chunks' factors exp(-(m_c - L_min) / lambda), from FP64, as pairs
    float2 Z;
    float Lmin;  // the minimum over the chunks' cost minima (combine_setup)
    int last;
};

// float-float helpers of the combine: a + b, and the product of two pairs (the
// high parts' rounding error by FMA, the cross terms; the lo * lo term is below
// the pairs' precision)
__device__ __forceinline__ float2 ff_sum(float2 a, float2 b) {
    ff_acc(a.x, a.y, b.x, b.y);
    return a;
}
__device__ __forceinline__ float2 ff_mul(float2 f, float2 v) {
    const float p = __fmul_rn(f.x, v.x);
    return make_float2(p, __fmaf_rn(f.x, v.y, __fmaf_rn(f.y, v.x, __fmaf_rn(f.x, v.x, -p))));
}

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

// CTA b's chunk of the 48 knot parameters: its row of the scratch gets S_c of
// the parameters, then z_c and m_c
__device__ __forceinline__ void chunk_partials(const UpdateArgs& a, int b, int G, double* rows, UpdSmem& s) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Dp = a.Dp;
    const int chunk = (a.n + G - 1) / G;
    const int k0 = b * chunk, k1 = min(a.n, k0 + chunk);
    // sum_k w_k U_k: warp w takes samples ks + w, ks + w + 8, ... of each
    // sub-chunk; lane i < 24 owns parameters 2i, 2i + 1.  The loads of the
    // warp's first UPD_PF samples go out first: they depend on neither the
    // costs' minimum nor the weights.
    const bool own = lane < UPD_TILE / 2;
    const float2* u2 = reinterpret_cast<const float2*>(a.U) + lane;
    const int ke0 = min(k1, k0 + UPD_SUB);
    float2 pf[UPD_PF];
#pragma unroll
    for (int q = 0; q < UPD_PF; q++) {
        const int k = k0 + warp + q * UPD_WARPS;
        pf[q] = own && k < ke0 ? __ldg(u2 + (size_t)k * (Dp / 2)) : make_float2(0.f, 0.f);
    }
    float lm = INFINITY;
    for (int k = k0 + tid; k < k1; k += UPD_THREADS) {
        const float l = __ldg(a.L + k);
        if (finitef(l)) lm = fminf(lm, l);
    }
    const float m = block_min(lm, s.red);
    const bool okc = finitef(m);
    float zs = 0.f, ze = 0.f;
    float s0 = 0.f, s1 = 0.f, e0 = 0.f, e1 = 0.f;
    if (okc)
        for (int ks = k0; ks < k1; ks += UPD_SUB) {
            // Eq. 1's weights around the chunk minimum, once per sample: exponent
            // and exp in FP64, kept as pairs
            const int k = ks + tid;
            float2 wk = make_float2(0.f, 0.f);
            if (k < k1) {
                const float l = __ldg(a.L + k);
                if (finitef(l)) {
                    const double wd = exp(-((double)l - (double)m) * a.inv_lambda);
                    wk.x = (float)wd;
                    wk.y = (float)(wd - (double)wk.x);
                }
            }
            ff_acc(zs, ze, wk.x, wk.y);
            __syncthreads();  // the previous sub-chunk's weights are consumed
            s.w[tid] = wk;
            __syncthreads();
            if (own) {
                int kb = ks + warp;
                if (ks == k0) {  // the prefetched samples, in the same order as the loop below
#pragma unroll
                    for (int q = 0; q < UPD_PF; q++) {
                        const int k = k0 + warp + q * UPD_WARPS;
                        if (k >= ke0) break;
                        const float2 wk = s.w[k - ks];
                        const float p0 = wk.x * pf[q].x, p1 = wk.x * pf[q].y;
                        ff_acc(s0, e0, p0, fmaf(wk.y, pf[q].x, fmaf(wk.x, pf[q].x, -p0)));
                        ff_acc(s1, e1, p1, fmaf(wk.y, pf[q].y, fmaf(wk.x, pf[q].y, -p1)));
                    }
                    kb = k0 + warp + UPD_PF * UPD_WARPS;
                }
                sum_chunk(s.w, ks, u2, Dp / 2, kb, min(k1, ks + UPD_SUB), s0, s1, e0, e1);
            }
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
    // the warps' pairs added in warp order; the row holds (hi, lo) pairs
    float2* row = reinterpret_cast<float2*>(rows) + (size_t)b * UPD_ROW;
    if (tid < UPD_TILE) {
        float2 v = s.part[0][tid];
        for (int w = 1; w < UPD_WARPS; w++) v = ff_sum(v, s.part[w][tid]);
        row[tid] = v;
    }
    if (tid == UPD_TILE) {
        float2 v = s.z[0];
        for (int w = 1; w < UPD_WARPS; w++) v = ff_sum(v, s.z[w]);
        row[UPD_TILE] = v;
    }
    if (tid == UPD_TILE + 1) row[UPD_TILE + 1] = make_float2(m, 0.f);
}

// publish this CTA's writes and count it in: true in the last of `total` CTAs
__device__ __forceinline__ bool count_in(unsigned* counter, unsigned total, UpdSmem& s) {
    return cta_count_in(counter, 1u, total, s.last);
}

// the last CTA: L_min over the G chunk minima, the factors f_c (FP64 exponent
// and exp, kept as pairs), and Z = sum_c f_c z_c in float-float (warp 0: lane j
// takes chunks j, j + 32, ..., then a fixed xor tree).  Returns whether any cost
// is finite.  The sums stay on the FP32 pipe: FP64 runs at 1/64 of its rate on
// this part, and its dependency chains cost more than the pairs' operations.
__device__ __forceinline__ bool combine_setup(const UpdateArgs& a, int G, const double* rows, UpdSmem& s) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2* row2 = reinterpret_cast<const float2*>(rows);
    constexpr int NQ = UPDATE_MAX_CTAS / 32;
    float2 zv[NQ];  // warp 0: the weight sums of chunks lane, lane + 32, ..., loaded with the minima
    if (warp == 0)
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int c = lane + 32 * q;
            zv[q] = c < G ? __ldcg(row2 + (size_t)c * UPD_ROW + UPD_TILE) : make_float2(0.f, 0.f);
        }
    const float mc = tid < G ? __ldcg(row2 + (size_t)tid * UPD_ROW + UPD_TILE + 1).x : INFINITY;
    const float Lmin = block_min(mc, s.red);
    const bool ok = finitef(Lmin);
    if (tid == 0) s.Lmin = Lmin;
    if (tid < G) {
        const double f = (ok && finitef(mc)) ? exp(-((double)mc - (double)Lmin) * a.inv_lambda) : 0.0;
        const float fh = (float)f;
        s.f[tid] = make_float2(fh, (float)(f - (double)fh));
    }
    __syncthreads();
    if (warp == 0) {
        float2 v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int c = lane + 32 * q;
            v[q] = c < G ? ff_mul(s.f[c], zv[q]) : make_float2(0.f, 0.f);
        }
        float2 z = ff_sum(ff_sum(v[0], v[1]), ff_sum(v[2], v[3]));
        static_assert(NQ == 4, "the tree above adds four chunks per lane");
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            z = ff_sum(z, make_float2(__shfl_xor_sync(0xffffffffu, z.x, o), __shfl_xor_sync(0xffffffffu, z.y, o)));
        if (lane == 0) s.Z = z;
    }
    __syncthreads();
    return ok;
}

// one round of a quad lane's chunk partials for parameter j: chunks c0, c0 + 4,
// ..., UPD_NB of them (zero past G)
__device__ __forceinline__ void load_round(float2 (&v)[UPD_NB], int G, const double* rows, int j, int c0) {
    const float2* row2 = reinterpret_cast<const float2*>(rows);
#pragma unroll
    for (int i = 0; i < UPD_NB; i++) {
        const int c = c0 + 4 * i;
        v[i] = c < G ? __ldcg(row2 + (size_t)c * UPD_ROW + j) : make_float2(0.f, 0.f);
    }
}

// S_j = sum_c f_c S_c[j] for tile parameter j by the 4 lanes q of a quad (chunks
// c = q mod 4, UPD_NB per round, each round's products added by a fixed pairwise
// tree, the rounds in order), added over the quad by a fixed xor tree,
// float-float throughout; every lane of the quad returns it.  v0 holds the first
// round (load_round(.., q)), loaded before the factors were formed.  The whole
// warp calls it.
__device__ __forceinline__ float2 combine_param(int G, const double* rows, int j, int q, const UpdSmem& s,
                                                const float2 (&v0)[UPD_NB]) {
    float2 acc = make_float2(0.f, 0.f);
    for (int c0 = q; c0 < G; c0 += 4 * UPD_NB) {
        float2 v[UPD_NB];
        if (c0 == q) {
#pragma unroll
            for (int i = 0; i < UPD_NB; i++) v[i] = v0[i];
        } else {
            load_round(v, G, rows, j, c0);
        }
#pragma unroll
        for (int i = 0; i < UPD_NB; i++) {
            const int c = c0 + 4 * i;
            v[i] = c < G ? ff_mul(s.f[c], v[i]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int span = 1; span < UPD_NB; span *= 2)
#pragma unroll
            for (int i = 0; i + span < UPD_NB; i += 2 * span) v[i] = ff_sum(v[i], v[i + span]);
        acc = ff_sum(acc, v[0]);
    }
    acc = ff_sum(acc, make_float2(__shfl_xor_sync(0xffffffffu, acc.x, 1), __shfl_xor_sync(0xffffffffu, acc.y, 1)));
    acc = ff_sum(acc, make_float2(__shfl_xor_sync(0xffffffffu, acc.x, 2), __shfl_xor_sync(0xffffffffu, acc.y, 2)));
    return acc;
}

// Knot representations (48 parameters): one parameter tile.
__global__ void __launch_bounds__(UPD_THREADS) k_update_knots(UpdateArgs a) {
    __shared__ UpdSmem s;
    __shared__ float s_mu[D];
    const int tid = threadIdx.x, G = gridDim.x;
    chunk_partials(a, blockIdx.x, G, a.part, s);
    if (!count_in(a.counter, (unsigned)G, s)) return;

    // last CTA: combine, apply, shift (the first round of partials loaded
    // before the factors are formed)
    const int j = tid >> 2, q = tid & 3;  // 64 quads, 48 parameters
    float2 v0[UPD_NB];
    load_round(v0, G, a.part, min(j, D - 1), q);
    const bool ok = combine_setup(a, G, a.part, s);
    {
        const float2 S = combine_param(G, a.part, min(j, D - 1), q, s, v0);
        if (j < D && q == 0) {
            // every cost non-finite: keep the previous mean
            const float mu_new = ok ? ff_div(S, s.Z) : a.mu[j];
            s_mu[j] = mu_new;
            if (a.mu_upd) a.mu_upd[j] = mu_new;
            if (j < NJ) a.u0[j] = mu_new;  // the spline at tau = 0 is knot 0
        }
    }
    if (tid == 0) {
        if (ok && a.wsum) *a.wsum = (double)s.Z.x + (double)s.Z.y;
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
    chunk_partials(a, blockIdx.x, G, a.part, s);
    if (!count_in(a.counter, (unsigned)G, s)) return;
    const int j = tid >> 2, q = tid & 3;
    float2 v0[UPD_NB];
    load_round(v0, G, a.part, min(j, D - 1), q);
    const bool ok = combine_setup(a, G, a.part, s);
    {
        const float2 S = combine_param(G, a.part, min(j, D - 1), q, s, v0);
        if (j < D && q == 0) a.partial_out[2 + j] = ok ? (double)S.x + (double)S.y : 0.0;
    }
    if (tid == 0) {
        a.partial_out[0] = (double)s.Lmin;
        a.partial_out[1] = ok ? (double)s.Z.x + (double)s.Z.y : 0.0;
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

// ---------------------------------------------------------------- direct targets

constexpr int ROW_GROUPS = 512;  // 16-byte parameter groups per column tile (threads per CTA at most)
constexpr int ROW_SUB = 256;     // samples whose weights sit in shared memory at a time
constexpr int ROW_NB = 8;        // rows whose loads a thread issues together
constexpr int ROW_MAX_CHUNKS = 512;
constexpr int CMB_THREADS = 512, CMB_WARPS = CMB_THREADS / 32;  // combine: 32 columns per CTA
constexpr int CMB_NB = 20;       // chunk partials a combining lane loads per round trip (one round: G <= 320)
static_assert(ROW_SUB % ROW_NB == 0, "a weight window holds whole batches");
static_assert(ROW_MAX_CHUNKS <= CMB_THREADS, "the combine loads one chunk's weight sum per thread");

static int row_tiles(int Dp) { return (Dp / 4 + ROW_GROUPS - 1) / ROW_GROUPS; }
static int row_groups(int Dp) {  // groups per tile: the tiles split the row evenly
    const int T = row_tiles(Dp);
    return (Dp / 4 + T - 1) / T;
}
int update_direct_chunks_cap(int Dp) {
    const int T = row_tiles(Dp), g = (1024 + T - 1) / T;
    return g < 1 ? 1 : (g > ROW_MAX_CHUNKS ? ROW_MAX_CHUNKS : g);
}
size_t update_direct_part_doubles(int Dp) { return (size_t)update_direct_chunks_cap(Dp) * (Dp + 1); }

// chunks of a direct-target update of n samples: about two CTAs per SM over the
// chunks and column tiles, at least 16 samples per chunk
static int update_direct_chunks(int n, int Dp, int sms) {
    const int T = row_tiles(Dp);
    int g = (2 * sms + T - 1) / T;
    g = min(g, (n + 15) / 16);
    g = min(g, update_direct_chunks_cap(Dp));
    return g < 1 ? 1 : g;
}

// The minimum over finite costs as an integer key for atomicMax: the float's
// bits made order-preserving as a signed integer (negative values have their
// magnitude bits flipped), then reversed as INT_MAX - key (modulo 2^32), so 0
// (the state between launches) means "no finite cost" -- no finite float maps
// there.
__device__ __forceinline__ unsigned lmin_key(float x) {
    const int i = __float_as_int(x);
    return 0x7fffffffu - (unsigned)(i >= 0 ? i : i ^ 0x7fffffff);
}
__device__ __forceinline__ float lmin_of_key(unsigned k) {
    const int i = (int)(0x7fffffffu - k);
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// (s, e) += v: Knuth's TwoSum of s + v, its error into e
__device__ __forceinline__ void ff_acc1(float& s, float& e, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
    s = t;
}
// (s, e) += w_a u_a + w_b u_b, the two products summed in FP32
__device__ __forceinline__ void ff_madd2(float& s, float& e, float wa, float ua, float wb, float ub) {
    ff_acc1(s, e, __fmaf_rn(wb, ub, __fmul_rn(wa, ua)));
}
__device__ __forceinline__ void ff_madd2_4(float (&s)[4], float (&e)[4], float wa, float4 a, float wb, float4 b) {
    ff_madd2(s[0], e[0], wa, a.x, wb, b.x);
    ff_madd2(s[1], e[1], wa, a.y, wb, b.y);
    ff_madd2(s[2], e[2], wa, a.z, wb, b.z);
    ff_madd2(s[3], e[3], wa, a.w, wb, b.w);
}

// minimum of v over the CTA's nw warps, returned to every thread
__device__ __forceinline__ float block_min_n(float v, float* red, int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();  // red is free
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = red[0];
    for (int w = 1; w < nw; w++) m = fminf(m, red[w]);
    return m;
}

// Programmatic dependent launch: the next kernel on the stream may start once
// every CTA of this one has called launch_dependents (or exited); a kernel
// launched that way waits in grid_dependency_wait until its predecessor has
// completed and its writes are visible.  Both are no-ops without the launch
// attribute.
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// L_min over the finite costs into counter[1] (the reversed key; 0 between
// launches): 4 costs per thread and round, loaded together
__global__ void __launch_bounds__(256) k_update_lmin(UpdateArgs a) {
    __shared__ float red[8];
    launch_dependents();  // the rows kernel's CTAs may start their loads of U now
    float lm = INFINITY;
    for (int k = blockIdx.x * 1024 + threadIdx.x; k < a.n; k += gridDim.x * 1024) {
        float l[4];
#pragma unroll
        for (int q = 0; q < 4; q++) l[q] = k + 256 * q < a.n ? __ldg(a.L + k + 256 * q) : INFINITY;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (finitef(l[q])) lm = fminf(lm, l[q]);
    }
    lm = block_min_n(lm, red, 8);
    if (threadIdx.x == 0 && finitef(lm)) atomicMax(a.counter + 1, lmin_key(lm));
}

// this thread's group of ROW_NB rows from row k (rows at or past k1 read nothing)
__device__ __forceinline__ void load_rows(float4 (&ub)[ROW_NB], const float4* u4, int D4, int k, int k1) {
#pragma unroll
    for (int q = 0; q < ROW_NB; q++)
        ub[q] = k + q < k1 ? __ldg(u4 + (size_t)(k + q) * D4) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// CTA (c, y): chunk c of the samples (contiguous, about n / G) against column
// tile y (W groups of 4 parameters).  Thread t owns group y W + t of every row.
// Its loads of the first ROW_NB rows go out before anything else; the weights
// of ROW_SUB samples at a time (exponent and exp in FP64 around L_min, rounded
// to FP32) sit in shared memory, and their float-float sum is kept.  Rows are
// added two at a time (one product, one FMA) into float-float sums, in order,
// ROW_NB rows' loads in flight.  Row c of the scratch (Dp + 1 float pairs) gets
// the tile's sums and, from tile 0, the chunk's weight sum z_c.
__global__ void __launch_bounds__(ROW_GROUPS) k_update_rows(UpdateArgs a, int W) {
    __shared__ float s_w[ROW_SUB];
    __shared__ float2 s_z[ROW_GROUPS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int c = blockIdx.x, G = gridDim.x, y = blockIdx.y;
    const int Dp = a.Dp, D4 = Dp >> 2;
    const int chunk = (a.n + G - 1) / G;
    const int k0 = min(a.n, c * chunk), k1 = min(a.n, k0 + chunk);
    const int g = y * W + tid;
    const bool own = tid < W && g < D4;
    const float4* u4 = reinterpret_cast<const float4*>(a.U) + g;
    float4 ub[ROW_NB];
    if (own) load_rows(ub, u4, D4, k0, k1);
    grid_dependency_wait();  // L_min is known once k_update_lmin has completed
    const unsigned key = __ldcg(a.counter + 1);
    const bool ok = key != 0u;
    const double m = ok ? (double)lmin_of_key(key) : 0.0;
    float sv[4] = {0.f, 0.f, 0.f, 0.f}, ev[4] = {0.f, 0.f, 0.f, 0.f};
    float zs = 0.f, ze = 0.f;
    for (int kb = k0; kb < k1; kb += ROW_NB) {
        const int ws = k0 + (kb - k0) / ROW_SUB * ROW_SUB;  // this weight window's first sample
        if (kb == ws) {
            __syncthreads();  // the previous window's weights are consumed
            const int nk = min(ROW_SUB, k1 - ws);
            for (int i = tid; i < nk; i += blockDim.x) {
                const float l = __ldg(a.L + ws + i);
                float wh = 0.f, wl = 0.f;
                if (ok && finitef(l)) {
                    const double wd = exp(-((double)l - m) * a.inv_lambda);
                    wh = (float)wd;
                    wl = (float)(wd - (double)wh);
                }
                s_w[i] = wh;
                ff_acc(zs, ze, wh, wl);
            }
            __syncthreads();
        }
        if (own) {
            if (kb != k0) load_rows(ub, u4, D4, kb, k1);
            const float* w = s_w + (kb - ws);
            if (kb + ROW_NB <= k1) {
#pragma unroll
                for (int q = 0; q < ROW_NB; q += 2) ff_madd2_4(sv, ev, w[q], ub[q], w[q + 1], ub[q + 1]);
            } else {
                const int nq = k1 - kb;  // 1 .. ROW_NB - 1; the rows past it loaded as zeros
#pragma unroll
                for (int q = 0; q < ROW_NB; q += 2)
                    if (q < nq) ff_madd2_4(sv, ev, w[q], ub[q], q + 1 < nq ? w[q + 1] : 0.f, ub[q + 1]);
            }
        }
    }
    launch_dependents();  // the combine may be scheduled while the last rows finish
    float2* row = reinterpret_cast<float2*>(a.part) + (size_t)c * (Dp + 1);
    if (own) {
#pragma unroll
        for (int i = 0; i < 4; i++) row[4 * g + i] = make_float2(sv[i], ev[i]);
    }
    if (y != 0) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, zs, o), ve = __shfl_xor_sync(0xffffffffu, ze, o);
        ff_acc(zs, ze, v, ve);
    }
    if (lane == 0) s_z[warp] = make_float2(zs, ze);
    __syncthreads();
    if (tid == 0) {
        float2 z = s_z[0];
        for (int w = 1; w < nw; w++) z = ff_sum(z, s_z[w]);
        row[Dp] = z;
    }
}

// The G chunk rows added per column in float-float: Z = sum_c z_c (chunk c by
// thread c, then a fixed tree over lanes and warps) and, for the CTA's 32
// columns, S_j = sum_c S_c[j] with warp w taking chunks c = w mod 16 (a fixed
// pairwise tree over its chunks, then over the 16 warps); mu' = S / Z, u0 = the
// first direct target, and the shift written straight from here: column
// (t, i) of mu' is the shifted nominal's column (t - ctrl_steps, i), and the
// last step's also fills the held steps past the end.  Pair arithmetic keeps
// the dependency chains on the FP32 pipe (FP64 runs at 1/64 of its rate here).
// With no finite cost (Z = 0, the same in every CTA) the previous mean is kept:
// every CTA copies its columns of it, and the last to count in shifts it.  CTA 0
// re-arms the L_min key (the rows kernel has read it).
__global__ void __launch_bounds__(CMB_THREADS) k_update_combine(UpdateArgs a, int G) {
    __shared__ float2 s_acc[CMB_WARPS][32];
    __shared__ float2 s_zw[CMB_WARPS];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Dp = a.Dp;
    const size_t RW = (size_t)Dp + 1;
    const float2* part = reinterpret_cast<const float2*>(a.part);
    grid_dependency_wait();  // every chunk row is written
    if (blockIdx.x == 0 && tid == 0) a.counter[1] = 0u;
    const int j = blockIdx.x * 32 + lane, jj = min(j, Dp - 1);
    const float2 zero = make_float2(0.f, 0.f);
    float2 z = tid < G ? __ldcg(part + tid * RW + Dp) : zero;
    float2 acc = zero;
    for (int c0 = warp; c0 < G; c0 += CMB_WARPS * CMB_NB) {
        float2 v[CMB_NB];
#pragma unroll
        for (int i = 0; i < CMB_NB; i++) {
            const int c = c0 + CMB_WARPS * i;
            v[i] = c < G ? __ldcg(part + c * RW + jj) : zero;
        }
#pragma unroll
        for (int span = 1; span < CMB_NB; span *= 2)
#pragma unroll
            for (int i = 0; i + span < CMB_NB; i += 2 * span) v[i] = ff_sum(v[i], v[i + span]);
        acc = ff_sum(acc, v[0]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        z = ff_sum(z, make_float2(__shfl_xor_sync(0xffffffffu, z.x, o), __shfl_xor_sync(0xffffffffu, z.y, o)));
    if (lane == 0) s_zw[warp] = z;
    s_acc[warp][lane] = acc;
    __syncthreads();
    // fixed trees over the 16 warps' sums (every warp forms Z; warp 0 the columns)
    float2 Zv[CMB_WARPS];
#pragma unroll
    for (int w = 0; w < CMB_WARPS; w++) Zv[w] = s_zw[w];
#pragma unroll
    for (int span = 1; span < CMB_WARPS; span *= 2)
#pragma unroll
        for (int i = 0; i + span < CMB_WARPS; i += 2 * span) Zv[i] = ff_sum(Zv[i], Zv[i + span]);
    const bool ok = Zv[0].x > 0.f;  // weights are >= 0: Z > 0 iff some cost is finite
    if (ok) {
        if (warp == 0) {
            float2 Sv[CMB_WARPS];
#pragma unroll
            for (int w = 0; w < CMB_WARPS; w++) Sv[w] = s_acc[w][lane];
#pragma unroll
            for (int span = 1; span < CMB_WARPS; span *= 2)
#pragma unroll
                for (int i = 0; i + span < CMB_WARPS; i += 2 * span) Sv[i] = ff_sum(Sv[i], Sv[i + span]);
            if (j < Dp) {
                const float mu_new = ff_div(Sv[0], Zv[0]);
                a.mu_upd[j] = mu_new;
                if (j < NJ) a.u0[j] = mu_new;  // the controls of step 0: the first direct target
                const int t = j / NJ, i = j % NJ, cs = a.ctrl_steps;
                if (t - cs >= 0 && t < a.H - 1) a.mu[(t - cs) * NJ + i] = mu_new;
                if (t == a.H - 1)
                    for (int td = max(0, t - cs); td < a.H; td++) a.mu[td * NJ + i] = mu_new;
            }
            if (blockIdx.x == 0 && lane == 0) {
                if (a.wsum) *a.wsum = (double)Zv[0].x + (double)Zv[0].y;
                if (a.status) *a.status = 0;
            }
        }
        return;
    }
    // no finite cost: keep the mean, then shift it once every CTA has read its columns
    if (warp == 0 && j < Dp) {
        const float mu_old = a.mu[j];
        a.mu_upd[j] = mu_old;
        if (j < NJ) a.u0[j] = mu_old;
    }
    if (blockIdx.x == 0 && tid == 0 && a.status) *a.status = 4;
    if (!cta_count_in(a.counter, 1u, gridDim.x, s_last)) return;
    for (int d = tid; d < Dp; d += CMB_THREADS) {
        const int t = d / NJ, i = d % NJ;
        const int src = min(t + a.ctrl_steps, a.H - 1);
        a.mu[d] = __ldcg(a.mu_upd + src * NJ + i);
    }
    if (tid == 0) a.counter[0] = 0u;  // re-arm for the next launch
}

int update_grid(int n) {
    int g = (n + 127) / 128;  // ~128 samples per CTA (measured: 64 per CTA costs 3 us more at n = 4096)
    return g < 1 ? 1 : (g > UPDATE_MAX_CTAS ? UPDATE_MAX_CTAS : g);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
    const bool direct = a.interp == INTERP_DIRECT;
    if (direct ? (a.Dp < 2 * NJ || a.Dp % NJ != 0 || !a.mu_upd || (reinterpret_cast<uintptr_t>(a.U) & 15u))
               : a.Dp != D)
        return cudaErrorInvalidValue;
    if (!direct) {
        k_update_knots<<<update_grid(a.n), UPD_THREADS, 0, st>>>(a);
    } else {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return cudaErrorInvalidValue;
        const int W = row_groups(a.Dp), G = update_direct_chunks(a.n, a.Dp, sms);
        k_update_lmin<<<max(1, min(2 * sms, (a.n + 1023) / 1024)), 256, 0, st>>>(a);
        // the rows and combine kernels as programmatic dependents of their predecessors
        cudaLaunchAttribute pdl[1];
        pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        pdl[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.stream = st;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(G, row_tiles(a.Dp));
        cfg.blockDim = dim3((W + 31) / 32 * 32);
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_update_rows, a, W);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3((a.Dp + 31) / 32);
        cfg.blockDim = dim3(CMB_THREADS);
        e = cudaLaunchKernelEx(&cfg, k_update_combine, a, G);
        if (e != cudaSuccess) return e;
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
