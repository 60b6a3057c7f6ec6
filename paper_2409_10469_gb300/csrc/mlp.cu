// mlp.cu -- the learned proposal network: a 62 -> 256 -> 256 -> 256 -> 48 MLP
// with GELU, BF16 weights and activations, FP32 accumulation, trained and run on
// the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// The paper leaves better sampling distributions to future work (arXiv
// 2409.10469, Sec. V-B) and cites learning one offline (Sec. II-B); this
// network maps a robot + task state to a mean for the spline knots.  It is
// trained on (state, updated mean) pairs from the plain controller and seeds
// half of the samples; plain MPPI's samples stay in every step.
//
// Every layer is one GEMM D = A B^T (A: M x K activations, B: N x K weights,
// both BF16, K-major) on tcgen05 with a fused epilogue.  The TMA-fed pipelined
// kernel of gemm.cu runs the forward layers and the whole backward pass: the
// epilogues also write transposed BF16 copies (activations H^T, gradients dZ^T)
// and the weights keep a transposed BF16 copy W^T, so every backward product
// reads K-major operands too: dH = dZ (W^T)^T, and dW = dZ^T (H^T)^T with K =
// the batch, cut into ranges whose partial sums are added in a fixed order.
// The thread-staged kernel below (k_gemm_tc: one 128 x NT tile per CTA,
// operands staged by the CTA's threads into the core-matrix layout of tc.cuh,
// one thread issuing the MMAs) remains for operands TMA cannot describe (rows
// not 16-byte aligned) through the raw GEMM entry point, and for the
// wait-timeout self-test.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/mppi.h"
#include "gemm.h"
#include "handle.h"
#include "memkind.h"
#include "tc.cuh"

using namespace mppi;

namespace mppi {

struct GemmArgs {
    const __nv_bfloat16* A;
    long a_sm, a_sk;  // A[m][k] = A[m * a_sm + k * a_sk]
    const __nv_bfloat16* B;
    long b_sn, b_sk;  // B[n][k] = B[n * b_sn + k * b_sk]
    int M, N, K;
    int epi;
    const float* bias;        // [N]
    const float* aux;         // pre-activation Z [M][ldaux] for EPI_GELU_BWD
    long ldaux;
    float* out;               // FP32 [M][ldo]
    long ldo;
    __nv_bfloat16* out_b;     // BF16 [M][ldob] (optional)
    long ldob;
    int vec_a, vec_b;         // stage with 16-byte loads (K-contiguous rows, K and strides multiples of 8, aligned)
    int* err;                 // set when a wait runs out
    uint32_t wait_limit;      // mbarrier polls before giving up (0 = default)
    int withhold_commit;      // self-test: never signal completion, so the wait runs out
};

template <int NT>
__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g) {
    static_assert(NT % 16 == 0 && NT >= 32 && NT <= 256, "tile width");
    constexpr uint32_t TCOLS = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                       // 128 x 64 bf16 = 16 KB
    unsigned char* sB = smem + 128 * tc::KCHUNK * 2;  // NT x 64 bf16
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;

    if (warp == 0) tc::tmem_alloc(&tmem_base, TCOLS);
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        s_fail = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::idesc_bf16_f32(128, NT);
    uint32_t phase = 0;
    const int nk = (g.K + tc::KCHUNK - 1) / tc::KCHUNK;
    for (int kc = 0; kc < nk; kc++) {
        const int k0 = kc * tc::KCHUNK;
        // stage A (128 x 64) and B (NT x 64), zero outside the matrices: 8 k-elements
        // (one 16-byte core-matrix row) per load when the rows are K-contiguous and
        // aligned, element by element otherwise (the transposed operands of backprop)
        if (g.vec_a) {
            // all loads of the chunk in flight before the first store (one memory round trip)
            constexpr int NA = 128 * (tc::KCHUNK / 8) / 128;
            uint4 v[NA];
#pragma unroll
            for (int i = 0; i < NA; i++) {
                const int idx = tid + 128 * i, r = idx >> 3, k = (idx & 7) * 8;
                const int gm = m0 + r, gk = k0 + k;
                v[i] = make_uint4(0u, 0u, 0u, 0u);
                if (gm < g.M && gk < g.K) v[i] = __ldg(reinterpret_cast<const uint4*>(g.A + (long)gm * g.a_sm + gk));
            }
#pragma unroll
            for (int i = 0; i < NA; i++) {
                const int idx = tid + 128 * i;
                *reinterpret_cast<uint4*>(sA + tc::tile_offset(idx >> 3, (idx & 7) * 8)) = v[i];
            }
        } else {
            for (int idx = tid; idx < 128 * tc::KCHUNK; idx += 128) {
                int r, k;
                if (g.a_sk == 1) { r = idx >> 6; k = idx & 63; } else { k = idx >> 7; r = idx & 127; }
                const int gm = m0 + r, gk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.f);
                if (gm < g.M && gk < g.K) v = g.A[(long)gm * g.a_sm + (long)gk * g.a_sk];
                *reinterpret_cast<__nv_bfloat16*>(sA + tc::tile_offset(r, k)) = v;
            }
        }
        if (g.vec_b) {
            constexpr int NB = NT * (tc::KCHUNK / 8) / 128;
            uint4 v[NB];
#pragma unroll
            for (int i = 0; i < NB; i++) {
                const int idx = tid + 128 * i, r = idx >> 3, k = (idx & 7) * 8;
                const int gn = n0 + r, gk = k0 + k;
                v[i] = make_uint4(0u, 0u, 0u, 0u);
                if (gn < g.N && gk < g.K) v[i] = __ldg(reinterpret_cast<const uint4*>(g.B + (long)gn * g.b_sn + gk));
            }
#pragma unroll
            for (int i = 0; i < NB; i++) {
                const int idx = tid + 128 * i;
                *reinterpret_cast<uint4*>(sB + tc::tile_offset(idx >> 3, (idx & 7) * 8)) = v[i];
            }
        } else {
            for (int idx = tid; idx < NT * tc::KCHUNK; idx += 128) {
                int r, k;
                if (g.b_sk == 1) { r = idx >> 6; k = idx & 63; } else { k = idx / NT; r = idx % NT; }
                const int gn = n0 + r, gk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.f);
                if (gn < g.N && gk < g.K) v = g.B[(long)gn * g.b_sn + (long)gk * g.b_sk];
                *reinterpret_cast<__nv_bfloat16*>(sB + tc::tile_offset(r, k)) = v;
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < tc::KCHUNK / 16; ks++) {
                const uint64_t ad = tc::smem_desc(a0 + ks * 2 * tc::CM_BYTES, tc::LBO, tc::SBO);
                const uint64_t bd = tc::smem_desc(b0 + ks * 2 * tc::CM_BYTES, tc::LBO, tc::SBO);
                if (!g.withhold_commit) tc::mma_bf16(tmem, ad, bd, idesc, (kc | ks) != 0);
            }
            if (!g.withhold_commit) tc::mma_commit(&bar);
        }
        // every thread waits for the MMAs (they read the staged tiles) before restaging
        if (!tc::mbar_wait(&bar, phase, g.wait_limit ? g.wait_limit : (1u << 22))) s_fail = 1;
        phase ^= 1u;
        __syncthreads();
        if (s_fail) break;
    }
    tc::fence_after();
    if (s_fail) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else {
        // epilogue: warp w owns rows 32w .. 32w + 31 (TMEM lanes)
        const int m = m0 + warp * 32 + lane;
        // 16-byte stores when a whole 16-column group is in range and the rows are aligned
        const bool vec_o = (g.ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.out) & 15u) == 0) &&
                           (!g.out_b || ((g.ldob % 8 == 0) && ((reinterpret_cast<uintptr_t>(g.out_b) & 15u) == 0)));
#pragma unroll 1
        for (int c = 0; c < NT / 16; c++) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
            if (m >= g.M) continue;
            const int nb = n0 + c * 16;
            if (vec_o && nb + 16 <= g.N) {
                float d[16], e[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    d[j] = v[j];
                    if (g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) d[j] += __ldg(g.bias + nb + j);
                    if (g.epi == EPI_GELU_BWD) d[j] *= gelu_grad(g.aux[(long)m * g.ldaux + nb + j]);
                    e[j] = g.epi == EPI_BIAS_GELU ? gelu(d[j]) : d[j];
                }
                float4* o4 = reinterpret_cast<float4*>(g.out + (long)m * g.ldo + nb);
#pragma unroll
                for (int q = 0; q < 4; q++) o4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
                if (g.out_b) {
                    uint4 pk[2];
                    __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(pk);
#pragma unroll
                    for (int q = 0; q < 8; q++) h2[q] = __floats2bfloat162_rn(e[2 * q], e[2 * q + 1]);
                    uint4* ob = reinterpret_cast<uint4*>(g.out_b + (long)m * g.ldob + nb);
                    ob[0] = pk[0];
                    ob[1] = pk[1];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int n = nb + j;
                    if (n >= g.N) break;
                    float d = v[j];
                    if (g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) d += g.bias[n];
                    if (g.epi == EPI_GELU_BWD) d *= gelu_grad(g.aux[(long)m * g.ldaux + n]);
                    g.out[(long)m * g.ldo + n] = d;
                    if (g.out_b) g.out_b[(long)m * g.ldob + n] = __float2bfloat16(g.epi == EPI_BIAS_GELU ? gelu(d) : d);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

static size_t gemm_smem(int nt) { return (size_t)(128 + nt) * tc::KCHUNK * 2; }

// 16-byte staging applies when every row of an operand starts on a 16-byte
// boundary and k runs along it, so every in-range 8-element group is whole
static bool vec_ok(const __nv_bfloat16* p, long s_row, long s_k, int K) {
    return s_k == 1 && K % 8 == 0 && s_row % 8 == 0 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

static cudaError_t launch_gemm(const GemmArgs& g0, cudaStream_t st) {
    GemmArgs g = g0;
    g.vec_a = vec_ok(g.A, g.a_sm, g.a_sk, g.K);
    g.vec_b = vec_ok(g.B, g.b_sn, g.b_sk, g.K);
    const int nt = g.N <= 64 ? 64 : 256;
    dim3 grid((g.M + 127) / 128, (g.N + nt - 1) / nt);
    if (nt == 64) {
        k_gemm_tc<64><<<grid, 128, gemm_smem(64), st>>>(g);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_gemm_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(256));
            attr = true;
        }
        k_gemm_tc<256><<<grid, 128, gemm_smem(256), st>>>(g);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise kernels

// FP32 [B][in] -> BF16 [B][ld] (zero padding past `in`), and optionally its
// transpose yt[c][r] (row stride ldt)
__global__ void k_to_bf16(const float* x, int B, int in, int ld, __nv_bfloat16* y, __nv_bfloat16* yt, long ldt) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)B * ld) return;
    const int r = (int)(i / ld), c = (int)(i % ld);
    const __nv_bfloat16 v = __float2bfloat16(c < in ? x[(long)r * in + c] : 0.f);
    if (y) y[i] = v;
    if (yt) yt[(long)c * ldt + r] = v;
}

// Small-batch forward on the CUDA cores (a control step's inference: a few
// robots' features).  A tensor-core tile is 128 rows, so a handful of samples
// would run mostly empty CTAs through four GEMM launches; and one CTA carrying
// them through all four layers waits on its 320 KB of weights one dependent
// load after another (40 us for one sample).  Here a cluster of SC_CL = 8 CTAs
// carries SB <= 8 samples (SB = 1, 2, 4 or 8, the fewest that hold them).
// CTA c owns rows [c R_l, (c + 1) R_l) of every layer's weights (R_l = 32, 32,
// 32, 6) and pulls all four slices (39 KB) into its shared memory with bulk
// copies at launch, so the weights cost one memory latency, spread over 8 SMs.
// Layer by layer, CTA c computes its R_l outputs of every sample and stores
// them into the activation buffer of all 8 CTAs (distributed shared memory, 4
// rows of a sample per 16-byte store); one cluster barrier separates layers.
// Thread (r, p) of a layer sums row r's dot product over k = 64 i + 4 p + {0..3}
// and 64 i + 32 + 4 p + {0..3} (so that 8 threads' 16-byte activation loads
// cover 128 contiguous bytes); three xor shuffles add the 8 parts.  With
// states as input instead of features, each CTA computes its samples'
// features (features.cuh) while the weights are in flight.  Rounding points as
// on the tensor-core path: BF16 inputs, BF16 weights, FP32 accumulation, FP32
// pre-activation + bias, BF16 of GELU for the next layer (held as FP32); the
// last layer's FP32 output is the result.
constexpr int SC_CL = 8;   // CTAs per cluster
constexpr int SC_T = 256;  // threads per CTA: 32 rows x 8 parts
__host__ __device__ constexpr int sc_k(int l) { return l == 0 ? 64 : 256; }   // input width (padded)
__host__ __device__ constexpr int sc_rows(int l) { return (l == 3 ? 48 : 256) / SC_CL; }
__host__ __device__ constexpr int sc_wofs(int l) { return l == 0 ? 0 : sc_wofs(l - 1) + sc_rows(l - 1) * sc_k(l - 1); }
constexpr int SC_WELEM = sc_wofs(4);  // a CTA's weight slices, BF16 elements
// dynamic shared memory: weights, two activation buffers [SB][256] FP32, 4 mbarriers
__host__ __device__ constexpr int sc_smem(int SB) { return SC_WELEM * 2 + 2 * SB * 256 * 4 + 4 * 8; }
static_assert(SC_WELEM * 2 % 16 == 0, "activation buffers 16-byte aligned");

struct SmallFwdArgs {
    const float* X;             // [B][62] features, or nullptr: computed from S
    const float* S;             // [B][lds] states
    int lds;
    FeatParams fp;
    int B;
    const __nv_bfloat16* W[4];  // [out][ld] BF16
    const float* bias[4];       // [out]
    float* Y;                   // [B][48]
    int* err;                   // set to 1 when a weight copy's wait runs out
    uint32_t wait_limit;        // mbarrier polls before giving up (0 = default)
    int withhold;               // self-test: layer 0's copy is never issued, so its waits run out
};

template <int SB>
__global__ void __cluster_dims__(SC_CL, 1, 1) __launch_bounds__(SC_T) k_mlp_cluster(SmallFwdArgs a) {
    extern __shared__ __align__(128) unsigned char sc_sm[];
    __nv_bfloat16* w_s = reinterpret_cast<__nv_bfloat16*>(sc_sm);
    float* h_s = reinterpret_cast<float*>(sc_sm + SC_WELEM * 2);  // [2][SB][256]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sc_sm + SC_WELEM * 2 + 2 * SB * 256 * 4);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t c = tc::cluster_rank();
    const int b0 = (blockIdx.x / SC_CL) * SB;
    const int nb = min(SB, a.B - b0);
    const int rl = lane >> 3, p = lane & 7, r = warp * 4 + rl;
    // warp 0 issues the weight copies first; the other warps meanwhile load
    // the given features (element i by thread 32 + i % 224) and every thread
    // its bias of each layer, all before anything waits on them
    constexpr int XW = SC_T - 32, XN = (SB * 64 + XW - 1) / XW;
    float xv[XN];
    float bias[4];
    if (warp != 0) {
#pragma unroll
        for (int j = 0; j < XN; j++) {
            const int i = t - 32 + j * XW, b = i >> 6, k = i & 63;
            xv[j] = (a.X && i < SB * 64 && b < nb && k < 62) ? __ldg(a.X + (size_t)(b0 + b) * 62 + k) : 0.f;
        }
    } else if (lane == 0) {
#pragma unroll
        for (int l = 0; l < 4; l++) tc::mbar_init_nofence(&bar[l], 1);
        tc::mbar_init_fence();
#pragma unroll
        for (int l = 0; l < 4; l++) {
            if (l == 0 && a.withhold) continue;
            const uint32_t bytes = sc_rows(l) * sc_k(l) * 2;
            tc::mbar_arrive_expect_tx(&bar[l], bytes);
            tc::bulk_load(tc::smem_u32(w_s + sc_wofs(l)), a.W[l] + (size_t)c * sc_rows(l) * sc_k(l), bytes, &bar[l]);
        }
    }
#pragma unroll
    for (int l = 0; l < 4; l++) bias[l] = __ldg(a.bias[l] + (int)c * sc_rows(l) + min(r, sc_rows(l) - 1));
    // layer-0 input: BF16-rounded features, zero past 62 and past the last sample
    if (a.X) {
        if (warp != 0) {
#pragma unroll
            for (int j = 0; j < XN; j++) {
                const int i = t - 32 + j * XW;
                if (i < SB * 64) h_s[(i >> 6) * 256 + (i & 63)] = __bfloat162float(__float2bfloat16(xv[j]));
            }
        }
    } else {
        float* f_s = h_s + SB * 256;  // [SB][62] in the second buffer, free until layer 0 writes it
        if (warp == 1 && lane < nb) state_features(a.S + (size_t)(b0 + lane) * a.lds, a.fp, f_s + lane * 62);
        __syncthreads();
        for (int i = t; i < SB * 64; i += SC_T) {
            const int b = i >> 6, k = i & 63;
            h_s[b * 256 + k] = __bfloat162float(__float2bfloat16(b < nb && k < 62 ? f_s[b * 62 + k] : 0.f));
        }
    }
    // the input is in place and the barriers' init visible to every thread;
    // the cluster barrier's wait (before layer 0's first remote store) then
    // finds every CTA started and done with its scratch
    __syncthreads();
    tc::cluster_arrive();
    const uint32_t lim = a.wait_limit ? a.wait_limit : (1u << 22);
    bool ok = true;
#pragma unroll
    for (int l = 0; l < 4; l++) {
        const int K = sc_k(l), R = sc_rows(l);
        const float* hin = h_s + (l & 1) * SB * 256;
        float* hout = h_s + ((l & 1) ^ 1) * SB * 256;
        if (!tc::mbar_wait(&bar[l], 0, lim)) ok = false;
        if (warp * 4 < R) {  // warp-uniform: the warp holds a row of this layer
            const __nv_bfloat16* wrow = w_s + sc_wofs(l) + min(r, R - 1) * K;
            float acc[SB];
#pragma unroll
            for (int b = 0; b < SB; b++) acc[b] = 0.f;
#pragma unroll
            for (int i = 0; i < K / 64; i++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    // odd row groups take the halves in the other order: the two
                    // rows of a half-warp then read different banks
                    const int k = 64 * i + 32 * (h ^ (rl & 1)) + 4 * p;
                    const uint2 wq = *reinterpret_cast<const uint2*>(wrow + k);
                    const float2 w01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wq.x));
                    const float2 w23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wq.y));
#pragma unroll
                    for (int b = 0; b < SB; b++) {
                        const float4 x = *reinterpret_cast<const float4*>(hin + b * 256 + k);
                        acc[b] = fmaf(w01.x, x.x, acc[b]);
                        acc[b] = fmaf(w01.y, x.y, acc[b]);
                        acc[b] = fmaf(w23.x, x.z, acc[b]);
                        acc[b] = fmaf(w23.y, x.w, acc[b]);
                    }
                }
            }
            // the 8 parts of row r are lanes 8 rl .. 8 rl + 7: after the
            // butterfly each of them holds all SB sums; lane p keeps sample p's
#pragma unroll
            for (int b = 0; b < SB; b++) {
                acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], 1);
                acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], 2);
                acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], 4);
            }
            float v = acc[0];
#pragma unroll
            for (int b = 1; b < SB; b++)
                if (p == b) v = acc[b];
            const int o = (int)c * R + min(r, R - 1);
            const float z = v + bias[l];
            if (l == 0) tc::cluster_wait();  // layer 0 has rows in every warp: all threads wait
            if (l < 3) {
                // (row rl, sample p) is on lane 8 rl + p: item (b, q) gathers the
                // warp's 4 rows of sample b and stores them into CTA q
                const float y = __bfloat162float(__float2bfloat16(gelu(z)));
#pragma unroll
                for (int i = 0; i < (SB * 8 + 31) / 32; i++) {
                    const int item = lane + 32 * i, b = min(item >> 3, SB - 1), q = item & 7;
                    float4 u;
                    u.x = __shfl_sync(0xffffffffu, y, b);
                    u.y = __shfl_sync(0xffffffffu, y, 8 + b);
                    u.z = __shfl_sync(0xffffffffu, y, 16 + b);
                    u.w = __shfl_sync(0xffffffffu, y, 24 + b);
                    if (item < SB * 8)
                        tc::st_cluster_v4(tc::cluster_map(tc::smem_u32(hout + b * 256 + (int)c * R + warp * 4), q), u);
                }
            } else if (r < R && p < nb) {
                a.Y[(size_t)(b0 + p) * 48 + o] = z;
            }
        }
        // layer l's outputs are in every CTA before layer l + 1 reads them, and
        // no CTA still reads the buffer layer l + 1 overwrites
        if (l < 3) tc::cluster_sync();
    }
    if (!ok) {
        atomicExch(a.err, 1);
        // the copies still in flight land before this CTA's shared memory is released
#pragma unroll
        for (int l = 0; l < 4; l++) tc::mbar_wait(&bar[l], 0, lim);
    }
}

// mean-squared error over B x O: loss and dY = 2 (Y - T) / (B O), FP32 and BF16
// [B][O], and the BF16 gradient transposed (dYt [O][ldt]).  One block of 256
// threads per MSE_ROWS samples: coalesced row-major reads and writes, the
// transposed copy through a shared tile (32 consecutive samples per row
// segment), the loss summed in the block and added once.
constexpr int MSE_ROWS = 32, MSE_MAXO = 64;
__global__ void __launch_bounds__(256) k_mse(const float* Y, const float* T, int B, int O, float scale, float* dY,
                                             __nv_bfloat16* dYb, __nv_bfloat16* dYt, long ldt, float* loss) {
    __shared__ __nv_bfloat16 tile[MSE_MAXO][MSE_ROWS + 2];
    __shared__ float red[8];
    const int b0 = blockIdx.x * MSE_ROWS, nb = min(MSE_ROWS, B - b0);
    float e = 0.f;
    for (int k = threadIdx.x; k < nb * O; k += blockDim.x) {
        const long i = (long)b0 * O + k;
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * scale;
        const __nv_bfloat16 h = __float2bfloat16(2.f * d * scale);
        dYb[i] = h;
        tile[k % O][k / O] = h;
        e += d * d * scale;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (dYt)
        for (int k = threadIdx.x; k < O * MSE_ROWS; k += blockDim.x) {
            const int o = k / MSE_ROWS, r = k % MSE_ROWS;
            if (r < nb) dYt[(long)o * ldt + b0 + r] = tile[o][r];
        }
    if (threadIdx.x == 0 && loss) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        atomicAdd(loss, t);
    }
}

// bias gradients: column sums of dZ [B][N] (row stride ld) in two fixed-order
// passes.  Pass 1: block (x, r) sums rows [r rows, (r + 1) rows) of columns
// 32 x .. 32 x + 31, warp w taking rows w, w + 8, ... (one coalesced 128-byte
// row segment per load), then the 8 warp sums in order -> part[r][n].
constexpr int COLSUM_SPLIT = 64;  // row ranges of pass 1 at most
__global__ void __launch_bounds__(256) k_colsum_part(const float* dZ, int B, int N, long ld, int rows, float* part) {
    __shared__ float s[8][33];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int n = blockIdx.x * 32 + lane, r = blockIdx.y;
    const int b0 = r * rows, b1 = min(B, b0 + rows);
    float acc = 0.f;
    if (n < N) {
#pragma unroll 4
        for (int b = b0 + w; b < b1; b += 8) acc += dZ[(long)b * ld + n];
    }
    s[w][lane] = acc;
    __syncthreads();
    if (w == 0 && n < N) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < 8; i++) t += s[i][lane];
        part[(long)r * N + n] = t;
    }
}
// Gradient finish of one layer, one thread per output:
//   i < M N:          dW[m][n] = sum over K ranges sp of part[sp][m][n], in order;
//   M N <= i < M N + M: db[m]  = sum over row ranges r of cpart[r][m], in order
// (the column-sum pass 2).
__global__ void k_grad_finish(const float* part, int nsplit, long sstride, int M, int N, long ldp, float* dw, long ldw,
                              const float* cpart, int R, float* db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.f;
    if (i < M * N) {
        const int m = i / N, n = i % N;
        const float* p = part + (long)m * ldp + n;
#pragma unroll 8
        for (int sp = 0; sp < nsplit; sp++) s += p[sp * sstride];
        dw[(long)m * ldw + n] = s;
    } else if (i < M * N + M) {
        const int m = i - M * N;
#pragma unroll 8
        for (int r = 0; r < R; r++) s += cpart[(long)r * M + m];
        db[m] = s;
    }
}

// AdamW on FP32 master parameters, refreshing the BF16 weight copies (W and W^T)
__global__ void k_adamw(float* p, const float* g, float* m1, float* m2, long n, float lr, float b1, float b2,
                        float eps, float wd, float c1, float c2, const long* wofs, const long* wlen,
                        __nv_bfloat16* const* wb, __nv_bfloat16* const* wbt, int nw, const int* wcols,
                        const int* wld) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float pi = p[i] - lr * ((a / c1) / (sqrtf(v / c2) + eps) + wd * p[i]);
    p[i] = pi;
    for (int w = 0; w < nw; w++)
        if (i >= wofs[w] && i < wofs[w] + wlen[w]) {
            const long j = i - wofs[w];
            const int r = (int)(j / wcols[w]), c = (int)(j % wcols[w]);
            const __nv_bfloat16 b = __float2bfloat16(pi);
            wb[w][(long)r * wld[w] + c] = b;
            if (wbt[w]) wbt[w][(long)c * (wlen[w] / wcols[w]) + r] = b;  // W^T [in][out]
        }
}

}  // namespace mppi

// ---------------------------------------------------------------- host object

namespace {

constexpr int IN = 62, IN_PAD = 64, HID = 256, OUT = 48;
constexpr int NL = 4;
constexpr int SMALL_BATCH = 128;  // forward batches up to this size run on the CUDA cores
constexpr int MAX_SPLIT = 64;     // K ranges of a weight-gradient product (partial sums buffered)
const int LIN[NL] = {IN, HID, HID, HID};
const int LOUT[NL] = {HID, HID, HID, OUT};
const int LLD[NL] = {IN_PAD, HID, HID, HID};  // leading dimension of each layer's BF16 input / weight rows

}  // namespace

struct mppi_mlp_s {
    int max_batch = 0;
    long nparam = 0;
    long wofs[NL], bofs[NL];
    float *d_p = nullptr, *d_g = nullptr, *d_m1 = nullptr, *d_m2 = nullptr;
    __nv_bfloat16* d_wb[NL] = {nullptr};      // BF16 weights [out][ld]
    __nv_bfloat16* d_hb[NL + 1] = {nullptr};  // BF16 activations: input [B][64], hidden [B][256]
    float* d_z[NL] = {nullptr};               // FP32 pre-activations [B][out]
    float* d_dz = nullptr;                    // FP32 dZ scratch [B][256]
    __nv_bfloat16* d_dzb = nullptr;           // BF16 dZ [B][256]
    __nv_bfloat16* d_dhb = nullptr;           // BF16 next dZ [B][256]
    float* d_dh = nullptr;                    // FP32 [B][256]
    float *d_T = nullptr, *d_X = nullptr, *d_loss = nullptr;
    int* d_err = nullptr;
    long *d_wofs = nullptr, *d_wlen = nullptr;
    int *d_wcols = nullptr, *d_wld = nullptr;
    __nv_bfloat16** d_wbp = nullptr;
    // K-major operands of the backward pass (ldt = batch capacity rounded up to 8)
    long ldt = 0;
    __nv_bfloat16* d_wbt[NL] = {nullptr};     // W^T [in][out] BF16 (layers 1..NL-1)
    __nv_bfloat16* d_ht[NL] = {nullptr};      // H^T of each layer's input [in padded][ldt]
    __nv_bfloat16* d_dzt[2] = {nullptr};      // dZ^T [256][ldt], two buffers
    float* d_part = nullptr;                  // split-K partial sums [MAX_SPLIT][256][256]
    float* d_cpart = nullptr;                 // bias-gradient partial column sums [COLSUM_SPLIT][256]
    __nv_bfloat16** d_wbtp = nullptr;
    int step = 0;
    int device = 0;  // the network's buffers live here
    std::string err;
};

static mppi_status mfail(mppi_mlp n, mppi_status s, const std::string& m) {
    if (n) n->err = m;
    return s;
}
#define MCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return mfail(net, MPPI_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// memory of the current device (or managed memory)
static bool mdev(const void* p) { return is_local(p); }

// the network's device is the current one and no buffer is another GPU's memory
static mppi_status local_call(mppi_mlp net, std::initializer_list<const void*> bufs) {
    const int dev = current_device();
    if (dev < 0) return mfail(net, MPPI_ERR_CUDA, "cudaGetDevice failed");
    if (dev != net->device) return mfail(net, MPPI_ERR_ARG, "the network's device is not the current device");
    if (any_foreign(dev, bufs)) return mfail(net, MPPI_ERR_ARG, "a buffer is memory of another GPU");
    return MPPI_OK;
}
#define MLP_LOCAL_CALL(...)                                              \
    do {                                                                 \
        const mppi_status s_ = local_call(net, {__VA_ARGS__});           \
        if (s_ != MPPI_OK) return s_;                                    \
    } while (0)

int mppi_mlp_device(mppi_mlp net) { return net->device; }

extern "C" mppi_status mppi_mlp_create(int max_batch, mppi_mlp* out) {
    if (!out || max_batch < 1) return MPPI_ERR_ARG;
    mppi_mlp net = new mppi_mlp_s();
    net->max_batch = max_batch;
    net->device = current_device();
    long o = 0;
    for (int l = 0; l < NL; l++) {
        net->wofs[l] = o;
        o += (long)LOUT[l] * LIN[l];
        net->bofs[l] = o;
        o += LOUT[l];
    }
    net->nparam = o;
    const long B = max_batch;
    bool ok = cudaMalloc((void**)&net->d_p, o * 4) == cudaSuccess && cudaMalloc((void**)&net->d_g, o * 4) == cudaSuccess &&
              cudaMalloc((void**)&net->d_m1, o * 4) == cudaSuccess && cudaMalloc((void**)&net->d_m2, o * 4) == cudaSuccess;
    for (int l = 0; ok && l < NL; l++) {
        ok = cudaMalloc((void**)&net->d_wb[l], (size_t)LOUT[l] * LLD[l] * 2) == cudaSuccess &&
             cudaMemset(net->d_wb[l], 0, (size_t)LOUT[l] * LLD[l] * 2) == cudaSuccess &&
             cudaMalloc((void**)&net->d_z[l], (size_t)B * LOUT[l] * 4) == cudaSuccess;
    }
    for (int l = 0; ok && l <= NL; l++) {
        const int w = l == 0 ? IN_PAD : (l == NL ? OUT : HID);
        ok = cudaMalloc((void**)&net->d_hb[l], (size_t)B * w * 2) == cudaSuccess;
    }
    ok = ok && cudaMalloc((void**)&net->d_dz, B * HID * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_dzb, B * HID * 2) == cudaSuccess &&
         cudaMalloc((void**)&net->d_dhb, B * HID * 2) == cudaSuccess &&
         cudaMalloc((void**)&net->d_dh, B * HID * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_T, B * OUT * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_X, B * IN * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_loss, 4) == cudaSuccess && cudaMalloc((void**)&net->d_err, 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_wofs, NL * 8) == cudaSuccess && cudaMalloc((void**)&net->d_wlen, NL * 8) == cudaSuccess &&
         cudaMalloc((void**)&net->d_wcols, NL * 4) == cudaSuccess && cudaMalloc((void**)&net->d_wld, NL * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_wbp, NL * sizeof(void*)) == cudaSuccess &&
         cudaMalloc((void**)&net->d_wbtp, NL * sizeof(void*)) == cudaSuccess &&
         cudaMalloc((void**)&net->d_part, (size_t)MAX_SPLIT * HID * HID * 4) == cudaSuccess &&
         cudaMalloc((void**)&net->d_cpart, (size_t)COLSUM_SPLIT * HID * 4) == cudaSuccess;
    net->ldt = (B + 7) / 8 * 8;
    for (int l = 0; ok && l < NL; l++) {
        if (l >= 1)
            ok = cudaMalloc((void**)&net->d_wbt[l], (size_t)LIN[l] * LOUT[l] * 2) == cudaSuccess;
        ok = ok && cudaMalloc((void**)&net->d_ht[l], (size_t)LLD[l] * net->ldt * 2) == cudaSuccess;
    }
    for (int i = 0; ok && i < 2; i++) ok = cudaMalloc((void**)&net->d_dzt[i], (size_t)HID * net->ldt * 2) == cudaSuccess;
    if (ok) {
        long wo[NL], wl[NL];
        int wc[NL], wd[NL];
        for (int l = 0; l < NL; l++) {
            wo[l] = net->wofs[l];
            wl[l] = (long)LOUT[l] * LIN[l];
            wc[l] = LIN[l];
            wd[l] = LLD[l];
        }
        ok = cudaMemcpy(net->d_wofs, wo, sizeof(wo), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(net->d_wlen, wl, sizeof(wl), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(net->d_wcols, wc, sizeof(wc), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(net->d_wld, wd, sizeof(wd), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(net->d_wbp, net->d_wb, sizeof(net->d_wb), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(net->d_wbtp, net->d_wbt, sizeof(net->d_wbt), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(net->d_m1, 0, o * 4) == cudaSuccess && cudaMemset(net->d_m2, 0, o * 4) == cudaSuccess &&
             cudaMemset(net->d_p, 0, o * 4) == cudaSuccess && cudaMemset(net->d_err, 0, 4) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        mppi_mlp_destroy(net);
        return MPPI_ERR_OOM;
    }
    *out = net;
    return MPPI_OK;
}

extern "C" mppi_status mppi_mlp_destroy(mppi_mlp net) {
    if (!net) return MPPI_ERR_ARG;
    cudaDeviceSynchronize();
    std::vector<void*> ps = {net->d_p, net->d_g, net->d_m1, net->d_m2, net->d_dz, net->d_dzb, net->d_dhb, net->d_dh,
                             net->d_T, net->d_X, net->d_loss, net->d_err, net->d_wofs, net->d_wlen, net->d_wcols,
                             net->d_wld, net->d_wbp, net->d_wbtp, net->d_part, net->d_cpart, net->d_dzt[0],
                             net->d_dzt[1]};
    for (int l = 0; l < NL; l++) {
        ps.push_back(net->d_wb[l]);
        ps.push_back(net->d_z[l]);
        ps.push_back(net->d_wbt[l]);
        ps.push_back(net->d_ht[l]);
    }
    for (int l = 0; l <= NL; l++) ps.push_back(net->d_hb[l]);
    for (void* p : ps)
        if (p) cudaFree(p);
    delete net;
    return MPPI_OK;
}

extern "C" const char* mppi_mlp_last_error(mppi_mlp net) { return net ? net->err.c_str() : "null mlp"; }

extern "C" long mppi_mlp_param_count(mppi_mlp net) { return net ? net->nparam : 0; }

// refresh every BF16 weight copy from the FP32 master parameters
static mppi_status refresh_bf16(mppi_mlp net, cudaStream_t st) {
    for (int l = 0; l < NL; l++) {
        const int rows = LOUT[l], cols = LIN[l], ld = LLD[l];
        // weights [rows][cols] FP32 -> [rows][ld] BF16 with zero padding
        k_to_bf16<<<(rows * ld + 255) / 256, 256, 0, st>>>(net->d_p + net->wofs[l], rows, cols, ld, net->d_wb[l],
                                                           net->d_wbt[l], rows);
        MCK(cudaGetLastError());
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_mlp_set_params(mppi_mlp net, const float* params, void* stream) {
    if (!net || !params) return MPPI_ERR_ARG;
    MLP_LOCAL_CALL(params);
    cudaStream_t st = (cudaStream_t)stream;
    MCK(cudaMemcpyAsync(net->d_p, params, net->nparam * 4, mdev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        st));
    MCK(cudaMemsetAsync(net->d_m1, 0, net->nparam * 4, st));
    MCK(cudaMemsetAsync(net->d_m2, 0, net->nparam * 4, st));
    net->step = 0;
    mppi_status s = refresh_bf16(net, st);
    if (s != MPPI_OK) return s;
    MCK(cudaStreamSynchronize(st));
    return MPPI_OK;
}

extern "C" mppi_status mppi_mlp_get_params(mppi_mlp net, float* params, void* stream) {
    if (!net || !params) return MPPI_ERR_ARG;
    MLP_LOCAL_CALL(params);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = mdev(params);
    MCK(cudaMemcpyAsync(params, net->d_p, net->nparam * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!dev) MCK(cudaStreamSynchronize(st));
    return MPPI_OK;
}

// one TMA-fed GEMM: A = a [M][K] (row stride lda), B = b [N][K] (row stride ldb)
static mppi_status tma_gemm(mppi_mlp net, TmaGemm& g, const __nv_bfloat16* a, long lda, const __nv_bfloat16* b,
                            long ldb, cudaStream_t st) {
    g.a = a;
    g.lda = lda;
    g.b = b;
    g.ldb = ldb;
    g.err = net->d_err;
    if (!gemm_tma_ok(g)) return mfail(net, MPPI_ERR_CUDA, "tensor-core GEMM operands break a TMA layout rule");
    MCK(launch_gemm_tma(g, st));
    return MPPI_OK;
}

static TmaGemm gemm_args(int M, int N, int K, int epi) {
    TmaGemm g;
    memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = N;
    g.K = K;
    g.nsplit = 1;
    g.epi = epi;
    return g;
}

// forward pass of B rows already converted to BF16 in d_hb[0]; outputs d_z[NL-1]
// (FP32); with `train` the hidden activations are also written transposed (H^T)
// for the weight gradients
static mppi_status forward_bf16(mppi_mlp net, int B, cudaStream_t st, bool train = false) {
    for (int l = 0; l < NL; l++) {
        const int ldi = (l == 0) ? IN_PAD : HID;
        TmaGemm g = gemm_args(B, LOUT[l], LLD[l], (l < NL - 1) ? EPI_BIAS_GELU : EPI_BIAS);
        g.bias = net->d_p + net->bofs[l];
        g.out = net->d_z[l];
        g.ldo = LOUT[l];
        if (l < NL - 1) {
            g.out_b = net->d_hb[l + 1];
            g.ldob = HID;
            if (train) {
                g.out_t = net->d_ht[l + 1];
                g.ldt = net->ldt;
            }
        }
        mppi_status s = tma_gemm(net, g, net->d_hb[l], ldi, net->d_wb[l], LLD[l], st);
        if (s != MPPI_OK) return s;
    }
    return MPPI_OK;
}

static mppi_status stage_x(mppi_mlp net, const float* X, int B, cudaStream_t st, bool train = false) {
    const float* dX = X;
    if (!mdev(X)) {
        MCK(cudaMemcpyAsync(net->d_X, X, (size_t)B * IN * 4, cudaMemcpyHostToDevice, st));
        dX = net->d_X;
    }
    k_to_bf16<<<(B * IN_PAD + 255) / 256, 256, 0, st>>>(dX, B, IN, IN_PAD, net->d_hb[0], train ? net->d_ht[0] : nullptr,
                                                         net->ldt);
    MCK(cudaGetLastError());
    return MPPI_OK;
}

static mppi_status check_err(mppi_mlp net, cudaStream_t st) {
    int e = 0;
    MCK(cudaMemcpyAsync(&e, net->d_err, 4, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    if (e) return mfail(net, MPPI_ERR_TIMEOUT, "a tensor-core wait ran out");
    return MPPI_OK;
}

template <int SB>
static cudaError_t launch_cluster(const SmallFwdArgs& a, int n, cudaStream_t st) {
    static bool attr = false;  // idempotent; set once per sample count
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_mlp_cluster<SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc_smem(SB));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_cluster<SB><<<SC_CL * ((n + SB - 1) / SB), SC_T, sc_smem(SB), st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_small(mppi_mlp net, const float* dX, const float* dS, int lds, const FeatParams* fp, int n,
                                float* dY, cudaStream_t st) {
    if (!net || n < 1 || n > SMALL_BATCH || n > net->max_batch) return cudaErrorInvalidValue;
    SmallFwdArgs a = {};
    a.X = dX;
    a.S = dS;
    a.lds = lds;
    if (fp) a.fp = *fp;
    a.B = n;
    for (int l = 0; l < NL; l++) {
        a.W[l] = net->d_wb[l];
        a.bias[l] = net->d_p + net->bofs[l];
    }
    a.Y = dY;
    a.err = net->d_err;
    if (n == 1) return launch_cluster<1>(a, n, st);
    if (n == 2) return launch_cluster<2>(a, n, st);
    if (n <= 4) return launch_cluster<4>(a, n, st);
    return launch_cluster<8>(a, n, st);
}

cudaError_t mppi_mlp_forward_small_dev(mppi_mlp net, const float* dX, int n, float* dY, cudaStream_t st) {
    return launch_small(net, dX, nullptr, 0, nullptr, n, dY, st);
}

cudaError_t mppi_mlp_forward_states_dev(mppi_mlp net, const float* dS, int lds, int n, const FeatParams& fp, float* dY,
                                        cudaStream_t st) {
    if (!dS || lds < fp.nx) return cudaErrorInvalidValue;
    return launch_small(net, nullptr, dS, lds, &fp, n, dY, st);
}

extern "C" mppi_status mppi_mlp_forward(mppi_mlp net, const float* X, int B, float* Y, void* stream) {
    if (!net || !X || !Y || B < 1 || B > net->max_batch) return MPPI_ERR_ARG;
    MLP_LOCAL_CALL(X, Y);
    cudaStream_t st = (cudaStream_t)stream;
    if (B <= SMALL_BATCH) {
        // a few samples: the fused CUDA-core forward (one launch)
        const float* dX = X;
        if (!mdev(X)) {
            MCK(cudaMemcpyAsync(net->d_X, X, (size_t)B * IN * 4, cudaMemcpyHostToDevice, st));
            dX = net->d_X;
        }
        const bool dev = mdev(Y);
        MCK(mppi_mlp_forward_small_dev(net, dX, B, dev ? Y : net->d_z[NL - 1], st));
        if (!dev) {
            MCK(cudaMemcpyAsync(Y, net->d_z[NL - 1], (size_t)B * OUT * 4, cudaMemcpyDeviceToHost, st));
            return check_err(net, st);
        }
        return MPPI_OK;
    }
    mppi_status s = stage_x(net, X, B, st);
    if (s == MPPI_OK) s = forward_bf16(net, B, st);
    if (s != MPPI_OK) return s;
    const bool dev = mdev(Y);
    MCK(cudaMemcpyAsync(Y, net->d_z[NL - 1], (size_t)B * OUT * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st));
    if (!dev) return check_err(net, st);
    return MPPI_OK;
}

extern "C" mppi_status mppi_mlp_train_step(mppi_mlp net, const float* X, const float* T, int B, float lr,
                                           float weight_decay, float* loss_out, float* grad_out, void* stream) {
    if (!net || !X || !T || B < 1 || B > net->max_batch) return MPPI_ERR_ARG;
    MLP_LOCAL_CALL(X, T, loss_out, grad_out);
    cudaStream_t st = (cudaStream_t)stream;
    mppi_status s = stage_x(net, X, B, st, true);
    if (s == MPPI_OK) s = forward_bf16(net, B, st, true);
    if (s != MPPI_OK) return s;
    const float* dT = T;
    if (!mdev(T)) {
        MCK(cudaMemcpyAsync(net->d_T, T, (size_t)B * OUT * 4, cudaMemcpyHostToDevice, st));
        dT = net->d_T;
    }
    MCK(cudaMemsetAsync(net->d_loss, 0, 4, st));
    const int n = B * OUT;
    int zt = 0;  // which dZ^T buffer holds the current layer's gradient
    static_assert(OUT <= MSE_MAXO, "output width of the loss tile");
    k_mse<<<(B + MSE_ROWS - 1) / MSE_ROWS, 256, 0, st>>>(net->d_z[NL - 1], dT, B, OUT, 1.f / (float)n, net->d_dz,
                                                          net->d_dzb, net->d_dzt[zt], net->ldt, net->d_loss);
    MCK(cudaGetLastError());
    // backward, layer NL-1 .. 0: dZ (FP32 d_dz and BF16 d_dzb [B][out], BF16 d_dzt[zt] [out][ldt])
    for (int l = NL - 1; l >= 0; l--) {
        const int out = LOUT[l], in = LIN[l];
        // dW[o][i] = sum_b dZ^T[o][b] H^T[i][b]: K = the batch, cut into ranges
        TmaGemm g = gemm_args(out, in, B, EPI_STORE);
        g.nsplit = gemm_tma_split(out, B, MAX_SPLIT);
        const int ldp = (in + 63) / 64 * 64;
        g.out = net->d_part;
        g.ldo = ldp;
        g.split_stride = (long)out * ldp;
        s = tma_gemm(net, g, net->d_dzt[zt], net->ldt, net->d_ht[l], net->ldt, st);
        if (s != MPPI_OK) return s;
        // bias gradient pass 1, then both sums of this layer in one launch
        const int R = std::min((B + 63) / 64, COLSUM_SPLIT), rows = (B + R - 1) / R;
        k_colsum_part<<<dim3((out + 31) / 32, R), dim3(32, 8), 0, st>>>(net->d_dz, B, out, out, rows, net->d_cpart);
        MCK(cudaGetLastError());
        k_grad_finish<<<(out * in + out + 255) / 256, 256, 0, st>>>(net->d_part, g.nsplit, g.split_stride, out, in, ldp,
                                                                   net->d_g + net->wofs[l], in, net->d_cpart, R,
                                                                   net->d_g + net->bofs[l]);
        MCK(cudaGetLastError());
        if (l == 0) break;
        // dH[b][i] = sum_o dZ[b][o] W^T[i][o], then dZ_prev = dH * gelu'(Z_prev)
        TmaGemm h = gemm_args(B, in, out, EPI_GELU_BWD);
        h.aux = net->d_z[l - 1];
        h.ldaux = HID;
        h.out = net->d_dh;
        h.ldo = HID;
        h.out_b = net->d_dhb;
        h.ldob = HID;
        h.out_t = net->d_dzt[zt ^ 1];
        h.ldt = net->ldt;
        s = tma_gemm(net, h, net->d_dzb, out, net->d_wbt[l], out, st);
        if (s != MPPI_OK) return s;
        std::swap(net->d_dz, net->d_dh);
        std::swap(net->d_dzb, net->d_dhb);
        zt ^= 1;
    }
    if (grad_out) {
        const bool dev = mdev(grad_out);
        MCK(cudaMemcpyAsync(grad_out, net->d_g, net->nparam * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (lr > 0.f) {
        net->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
        k_adamw<<<(int)((net->nparam + 255) / 256), 256, 0, st>>>(net->d_p, net->d_g, net->d_m1, net->d_m2, net->nparam,
                                                                  lr, b1, b2, 1e-8f, weight_decay, c1, c2, net->d_wofs,
                                                                  net->d_wlen, net->d_wbp, net->d_wbtp, NL, net->d_wcols,
                                                                  net->d_wld);
        MCK(cudaGetLastError());
    }
    if (loss_out) {
        const bool dev = mdev(loss_out);
        MCK(cudaMemcpyAsync(loss_out, net->d_loss, 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        if (!dev) return check_err(net, st);
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                                         void* stream) {
    if (!A || !B || !D || M < 1 || N < 1 || N > 256 || K < 1) return MPPI_ERR_ARG;
    if (!mdev(A) || !mdev(B) || !mdev(D)) return MPPI_ERR_ARG;
    // the wait-timeout flag: one per device for the process, allocated on first use
    static int* err_flag[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MPPI_ERR_CUDA;
    if (!err_flag[dev] && cudaMalloc((void**)&err_flag[dev], 4) != cudaSuccess) {
        err_flag[dev] = nullptr;
        return MPPI_ERR_OOM;
    }
    int* err = err_flag[dev];
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(err, 0, 4, st);
    // TMA-fed pipeline when both operands' rows start on 16-byte boundaries
    TmaGemm t;
    memset(&t, 0, sizeof(t));
    t.M = M;
    t.N = N;
    t.K = K;
    t.nsplit = 1;
    t.epi = EPI_STORE;
    t.out = D;
    t.ldo = N;
    t.err = err;
    t.a = reinterpret_cast<const __nv_bfloat16*>(A);
    t.lda = K;
    t.b = reinterpret_cast<const __nv_bfloat16*>(B);
    t.ldb = K;
    if (N % 4 == 0 && gemm_tma_ok(t)) {
        cudaError_t e = launch_gemm_tma(t, st);
        int h = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return MPPI_ERR_CUDA;
        return h ? MPPI_ERR_TIMEOUT : MPPI_OK;
    }
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = reinterpret_cast<const __nv_bfloat16*>(A);
    g.a_sm = K;
    g.a_sk = 1;
    g.B = reinterpret_cast<const __nv_bfloat16*>(B);
    g.b_sn = K;
    g.b_sk = 1;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = EPI_STORE;
    g.out = D;
    g.ldo = N;
    g.err = err;
    cudaError_t e = launch_gemm(g, st);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    return h ? MPPI_ERR_TIMEOUT : MPPI_OK;
}

extern "C" mppi_status mppi_selftest_wait_timeout(void* stream) {
    // a 128 x 64 x 64 GEMM whose completion is never signalled, on both
    // tensor-core kernels: the bounded mbarrier waits must run out, each kernel
    // must record it, drain its copies, free its tensor memory and return, and
    // the context must stay usable; then the same for the cluster forward
    cudaStream_t st = (cudaStream_t)stream;
    __nv_bfloat16 *A = nullptr, *B = nullptr;
    float* D = nullptr;
    int* err = nullptr;
    if (cudaMalloc((void**)&A, 128 * 64 * 2) != cudaSuccess || cudaMalloc((void**)&B, 64 * 64 * 2) != cudaSuccess ||
        cudaMalloc((void**)&D, 128 * 64 * 4) != cudaSuccess || cudaMalloc((void**)&err, 4) != cudaSuccess) {
        cudaFree(A); cudaFree(B); cudaFree(D); cudaFree(err);
        return MPPI_ERR_OOM;
    }
    cudaMemsetAsync(A, 0, 128 * 64 * 2, st);
    cudaMemsetAsync(B, 0, 64 * 64 * 2, st);
    cudaMemsetAsync(err, 0, 4, st);
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = A; g.a_sm = 64; g.a_sk = 1;
    g.B = B; g.b_sn = 64; g.b_sk = 1;
    g.M = 128; g.N = 64; g.K = 64;
    g.epi = EPI_STORE; g.out = D; g.ldo = 64; g.err = err;
    g.wait_limit = 1u << 12;
    g.withhold_commit = 1;
    cudaError_t e = launch_gemm(g, st);
    int h = 0, h2 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // the same on the TMA-fed kernel
    TmaGemm t;
    memset(&t, 0, sizeof(t));
    t.M = 128; t.N = 64; t.K = 64; t.nsplit = 1;
    t.epi = EPI_STORE; t.out = D; t.ldo = 64; t.err = err;
    t.wait_limit = 1u << 12;
    t.withhold_commit = 1;
    t.a = A; t.lda = 64; t.b = B; t.ldb = 64;
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, st);
    if (e == cudaSuccess) e = launch_gemm_tma(t, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h2, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // the cluster forward with its first layer's weight copy withheld: every
    // thread's wait on that layer runs out, the kernel records it, keeps in step
    // with its cluster's barriers and returns
    int h3 = 0;
    unsigned char* buf = nullptr;
    const size_t wbytes = ((size_t)HID * IN_PAD + 2 * (size_t)HID * HID + (size_t)OUT * HID) * 2;
    const size_t bytes = wbytes + (3 * HID + OUT) * 4 + 64 * 4 + 64 * 4;
    if (e == cudaSuccess) e = cudaMalloc((void**)&buf, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, st);
    if (e == cudaSuccess) {
        SmallFwdArgs c = {};
        size_t o = 0;
        for (int l = 0; l < NL; l++) {
            c.W[l] = reinterpret_cast<const __nv_bfloat16*>(buf + o);
            o += (size_t)LOUT[l] * LLD[l] * 2;
        }
        for (int l = 0; l < NL; l++) {
            c.bias[l] = reinterpret_cast<const float*>(buf + o);
            o += (size_t)LOUT[l] * 4;
        }
        c.X = reinterpret_cast<const float*>(buf + o);
        c.Y = reinterpret_cast<float*>(buf + o + 64 * 4);
        c.B = 1;
        c.err = err;
        c.wait_limit = 1u << 12;
        c.withhold = 1;
        e = launch_cluster<1>(c, 1, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h3, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(A); cudaFree(B); cudaFree(D); cudaFree(err); cudaFree(buf);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    return (h && h2 && h3) ? MPPI_ERR_TIMEOUT : MPPI_OK;
}
