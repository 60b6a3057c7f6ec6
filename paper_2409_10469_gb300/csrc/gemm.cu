// gemm.cu -- BF16 x BF16 -> FP32 GEMM D = A B^T on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), fed by TMA, for the proposal network's
// layers, its backward pass and the raw GEMM entry point.
//
// One persistent CTA per SM walks output tiles of 128 rows x NT columns (for the
// weight gradients: tiles x ranges of K).  The warps have fixed roles:
//   warp 0     TMA producer: 64-wide K chunks of A (128 rows) and B (NT rows)
//              into a ring of 128-byte-swizzled shared-memory slots (3 deep for
//              NT = 256 and 128, 4 for NT = 64);
//   warp 1     allocates 2 x NT TMEM columns (two accumulators); one lane issues
//              the tcgen05.mma of every chunk and frees the ring slot with
//              tcgen05.commit, then hands the finished accumulator on the same way;
//   warps 2-9  epilogue: warp w reads TMEM lane quarter w % 4 (the quarter its
//              position in the warpgroup may access) and one half of the columns,
//              applies bias / GELU / GELU', writes the transposed BF16 copy the
//              backward pass reads K-major, and stages the row-major outputs in
//              swizzled shared-memory blocks that TMA bulk stores write out;
//              then frees the accumulator.
// So the loads of the next chunks, the MMAs of chunk i and the epilogue of
// the previous tile run at the same time.  Every mbarrier wait has an iteration
// limit; a wait that runs out sets the error flag, and each role drains what
// it has in flight (its TMA loads, its MMAs) before the CTA frees TMEM and exits.
#include "gemm.h"

#include <mutex>

#include "tc.cuh"

namespace mppi {

constexpr int GT_EPI_WARPS = 8;
constexpr int GT_THREADS = 32 * (2 + GT_EPI_WARPS);
constexpr uint32_t GT_A_BYTES = 128 * 64 * 2;
// one epilogue warp's staging buffer: a 32 x 32 FP32 block (128-byte rows,
// 128-byte swizzle), a 32 x 32 BF16 block (64-byte rows, 64-byte swizzle) and
// the transposed 32 x 32 BF16 block (rows = columns n, 64 bytes of rows m, no
// swizzle), the layouts the output tensor maps' TMA stores read
constexpr uint32_t GT_STG_F32 = 32 * 128;
constexpr uint32_t GT_STG_T = GT_STG_F32 + 32 * 64;
constexpr uint32_t GT_STG_BUF = GT_STG_T + 32 * 64;      // 8 KB, a multiple of 1024

// Shared memory within 227 KB: for NT = 256 three ring stages (the weights are
// reloaded for every tile, so the loads need the depth: measured 22 us against
// 27 us with two stages and double staging at 65536 x 256 x 256) and one
// staging buffer per warp; for NT = 128 three stages and for NT = 64 four, both
// with two staging buffers used by alternate chunks, so a chunk waits only for
// the store two chunks back.
template <int NT>
struct GtCfg {
    static constexpr int STAGES = NT == 64 ? 4 : 3;
    static constexpr int NBUF = NT == 256 ? 1 : 2;
    static constexpr uint32_t STAGE = GT_A_BYTES + NT * 64 * 2;  // a multiple of 1024
    static constexpr uint32_t STG_BYTES = NBUF * GT_STG_BUF;
    static constexpr uint32_t SMEM = STAGES * STAGE + GT_EPI_WARPS * STG_BYTES + 1024;  // + alignment slack
    static constexpr uint32_t TCOLS = 2 * NT;
};

__device__ __forceinline__ void gt_fail(const TmaGemm& g, volatile int* s_fail) {
    *s_fail = 1;
    if (g.err) atomicExch(g.err, 1);
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled block of 128-byte
// rows (chunk index XOR row % 8), and in a 64-byte-swizzled block of 64-byte rows
// (chunk index XOR (row / 2) % 4); both are bank-conflict free when 8 consecutive
// lanes write the same chunk of 8 consecutive rows, or 8 chunks of one row
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }
__device__ __forceinline__ uint32_t sw64(int r, int c) { return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4)); }

// Epilogue of a warp's 32 x 32 block: rows m0 .. m0 + 31 (lane = row in v, as
// tcgen05.ld delivers it), columns nb .. nb + 31 (nb < N) of K range sp.  The
// arithmetic runs in that row-per-lane layout, which also fills the transposed
// block (lanes = consecutive rows, so each row of it is written whole).  The
// outputs go to the warp's staging blocks and leave by TMA bulk stores issued
// by lane 0 (which clip rows >= M and columns >= N); the GELU' input aux comes
// in through the FP32 block.  Before the buffer is written, lane 0 waits until the
// store that used it last (NBUF chunks back: one group per chunk) has read it.
template <int NBUF>
__device__ __forceinline__ void gt_epilogue(const TmaGemm& g, int m0, int nb, int sp, const float (&v)[32],
                                            unsigned char* S, uint32_t s_addr, int lane) {
    const int ncol = min(32, g.N - nb);
    const bool bias = g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU;
    if (lane == 0) tc::bulk_wait_read<NBUF - 1>();
    __syncwarp();
    float d[32];
#pragma unroll
    for (int j = 0; j < 32; j++) d[j] = v[j];
    if (bias) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (nb + 4 * q + 4 <= g.N) {
                const float4 b = __ldg(reinterpret_cast<const float4*>(g.bias + nb) + q);
                d[4 * q] += b.x;
                d[4 * q + 1] += b.y;
                d[4 * q + 2] += b.z;
                d[4 * q + 3] += b.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (4 * q + k < ncol) d[4 * q + k] += g.bias[nb + 4 * q + k];
            }
        }
    }
    if (g.epi == EPI_GELU_BWD) {
        // aux read coalesced (8 lanes x 16 B per row) into the FP32 block, then each lane takes its row
        const int c = lane & 7;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int r = (lane >> 3) + 4 * i, mr = m0 + r;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mr < g.M) {
                const float* src = g.aux + (long)mr * g.ldaux + nb + 4 * c;
                if (4 * c + 4 <= ncol) {
                    a = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    if (4 * c < ncol) a.x = src[0];
                    if (4 * c + 1 < ncol) a.y = src[1];
                    if (4 * c + 2 < ncol) a.z = src[2];
                }
            }
            *reinterpret_cast<float4*>(S + sw128(r, c)) = a;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 z = *reinterpret_cast<const float4*>(S + sw128(lane, q));
            d[4 * q] *= gelu_grad(z.x);
            d[4 * q + 1] *= gelu_grad(z.y);
            d[4 * q + 2] *= gelu_grad(z.z);
            d[4 * q + 3] *= gelu_grad(z.w);
        }
        __syncwarp();
    }
    __nv_bfloat162 h2[16];
    if (g.out_b || g.out_t) {
#pragma unroll
        for (int q = 0; q < 16; q++) {
            float a = d[2 * q], b = d[2 * q + 1];
            if (g.epi == EPI_BIAS_GELU) {
                a = gelu(a);
                b = gelu(b);
            }
            h2[q] = __floats2bfloat162_rn(a, b);
        }
    }
    if (g.out_t) {
        // transposed block: row n holds the 32 rows m of column n (lanes write 64
        // contiguous bytes per row; columns >= N and rows >= M are clipped by the store)
        __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(S + GT_STG_T);
#pragma unroll
        for (int q = 0; q < 16; q++) {
            T[(2 * q) * 32 + lane] = h2[q].x;
            T[(2 * q + 1) * 32 + lane] = h2[q].y;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; q++)
        *reinterpret_cast<float4*>(S + sw128(lane, q)) = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
    if (g.out_b) {
        const uint4* src = reinterpret_cast<const uint4*>(h2);
#pragma unroll
        for (int q = 0; q < 4; q++) *reinterpret_cast<uint4*>(S + GT_STG_F32 + sw64(lane, q)) = src[q];
    }
    tc::fence_proxy_async();  // the generic-proxy writes above become visible to the TMA unit
    __syncwarp();
    if (lane == 0) {
        if (m0 < g.M) {
            tc::tma_store_3d(&g.to, nb, m0, sp, s_addr);
            if (g.out_b) tc::tma_store_2d(&g.tob, nb, m0, s_addr + GT_STG_F32);
            if (g.out_t) tc::tma_store_2d(&g.tot, m0, nb, s_addr + GT_STG_T);
        }
        tc::bulk_commit();  // one group per chunk, empty for rows past M
    }
}

template <int NT>
__global__ void __launch_bounds__(GT_THREADS, 1) k_gemm_tma(const __grid_constant__ TmaGemm g) {
    using Cfg = GtCfg<NT>;
    extern __shared__ unsigned char gt_smem[];
    __shared__ __align__(8) uint64_t full[GtCfg<NT>::STAGES], empty[GtCfg<NT>::STAGES], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ring = (tc::smem_u32(gt_smem) + 1023u) & ~1023u;
    const uint32_t lim = g.wait_limit ? g.wait_limit : (1u << 22);
    const int mtiles = (g.M + 127) / 128, nk = (g.K + 63) / 64;
    const int kcs = g.kcs;
    // work unit u: K range u % nsplit of column tile (u / nsplit) % ntiles of row tile u / (nsplit ntiles)
    const int units = mtiles * g.ntiles * g.nsplit;

    if (warp == 1) tc::tmem_alloc(&tmem_base, Cfg::TCOLS);
    if (tid == 0) {
        for (int s = 0; s < Cfg::STAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], GT_EPI_WARPS);
        }
        tc::mbar_init(&drain, 1);
        s_fail = 0;
    }
    if (tid == 32) {
        tc::tma_prefetch_desc(&g.ta);
        tc::tma_prefetch_desc(&g.tb);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer
            uint32_t it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                const int sp = u % g.nsplit, nt = (u / g.nsplit) % g.ntiles, mt = u / (g.nsplit * g.ntiles);
                const int kb = sp * kcs, ke = min(nk, kb + kcs);
                for (int kc = kb; kc < ke; kc++) {
                    const uint32_t s = it % Cfg::STAGES, ph = (it / Cfg::STAGES) & 1u;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, lim) || s_fail) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = ring + s * Cfg::STAGE;
                    tc::mbar_arrive_expect_tx(&full[s], Cfg::STAGE);
                    tc::tma_load_2d(sa, &g.ta, kc * 64, mt * 128, &full[s]);
                    tc::tma_load_2d(sa + GT_A_BYTES, &g.tb, kc * 64, nt * NT, &full[s]);
                    it++;
                }
            }
            if (!ok) gt_fail(g, &s_fail);
            // every load issued must land before the CTA may exit
            for (uint32_t s = 0; s < Cfg::STAGES && s < it; s++) {
                const uint32_t last = it - 1u - ((it - 1u - s) % Cfg::STAGES);  // last issue into slot s
                if (!tc::mbar_wait(&full[s], (last / Cfg::STAGES) & 1u, lim)) gt_fail(g, &s_fail);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = tc::idesc_bf16_f32(128, NT);
            uint32_t it = 0, j = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x, j++) {
                const int sp = u % g.nsplit;
                const int kb = sp * kcs, ke = min(nk, kb + kcs);
                const uint32_t acc = j & 1u, aph = (j >> 1) & 1u;
                if (!tc::mbar_wait(&tempty[acc], aph ^ 1u, lim) || s_fail) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t d = tmem + acc * NT;
                for (int kc = kb; kc < ke; kc++) {
                    const uint32_t s = it % Cfg::STAGES, ph = (it / Cfg::STAGES) & 1u;
                    if (!tc::mbar_wait(&full[s], ph, lim) || s_fail) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t sa = ring + s * Cfg::STAGE;
                    const uint64_t ad = tc::smem_desc_sw128(sa), bd = tc::smem_desc_sw128(sa + GT_A_BYTES);
                    if (!g.withhold_commit) {
#pragma unroll
                        for (int ks = 0; ks < 4; ks++)
                            tc::mma_bf16(d, ad + 2u * ks, bd + 2u * ks, idesc, (kc > kb || ks > 0) ? 1u : 0u);
                        tc::mma_commit(&empty[s]);
                    }
                    it++;
                }
                if (!ok) break;
                if (!g.withhold_commit) tc::mma_commit(&tfull[acc]);
            }
            if (!ok) gt_fail(g, &s_fail);
            // the MMAs read the ring and write TMEM until they complete
            tc::mma_commit(&drain);
            if (!tc::mbar_wait(&drain, 0, lim)) gt_fail(g, &s_fail);
        }
    } else {
        // ---- epilogue
        const int q = warp & 3, hf = (warp - 2) >> 2;
        const uint32_t s_addr = ring + Cfg::STAGES * Cfg::STAGE + (warp - 2) * Cfg::STG_BYTES;
        unsigned char* stg = gt_smem + (s_addr - tc::smem_u32(gt_smem));
        uint32_t j = 0, nchunk = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, j++) {
            const int sp = u % g.nsplit, nt = (u / g.nsplit) % g.ntiles, mt = u / (g.nsplit * g.ntiles);
            const uint32_t acc = j & 1u, aph = (j >> 1) & 1u;
            int ok = 0;
            if (lane == 0) ok = tc::mbar_wait(&tfull[acc], aph, lim) && !s_fail;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) gt_fail(g, &s_fail);
                break;
            }
            __syncwarp();
            tc::fence_after();
            const int m0 = mt * 128 + q * 32;
#pragma unroll 1
            for (int c = 0; c < NT / 2; c += 32) {
                const int cb = hf * (NT / 2) + c, nb = nt * NT + cb;
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * NT + (uint32_t)cb, v);
                if (nb < g.N) {
                    const uint32_t o = (nchunk++ % Cfg::NBUF) * GT_STG_BUF;
                    gt_epilogue<Cfg::NBUF>(g, m0, nb, sp, v, stg + o, s_addr + o, lane);
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[acc]);
        }
        // the bulk stores read the staging blocks and write global memory until they complete
        if (lane == 0) tc::bulk_wait_all();
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, Cfg::TCOLS);
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// rank 2 or 3 map: dims[0] contiguous, strides in bytes for dims 1 .. rank-1
static bool encode(CUtensorMap* tm, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
                   const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle sw) {
    EncodeTiledFn f = encoder();
    if (!f || !base || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
    for (int i = 0; i < rank - 1; i++)
        if (strides[i] % 16) return false;
    const cuuint32_t es[3] = {1, 1, 1};
    return f(tm, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encode_kmajor(CUtensorMap* tm, const void* base, long rows, long K, long ld, int box_rows) {
    if (rows < 1 || K < 1 || ld < K || box_rows < 1 || box_rows > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

// the epilogue's store maps: out as [nsplit][M][ldo] FP32, out_b as [M][ldob]
// BF16 and out_t as [N][ldt] BF16, boxes of 32 x 32 in the staging blocks' layouts
static bool encode_outputs(TmaGemm& g) {
    const long sst = g.nsplit > 1 ? g.split_stride : (long)g.M * g.ldo;
    const cuuint64_t d3[3] = {(cuuint64_t)g.N, (cuuint64_t)g.M, (cuuint64_t)g.nsplit};
    const cuuint64_t s3[2] = {(cuuint64_t)g.ldo * 4, (cuuint64_t)sst * 4};
    const cuuint32_t b3[3] = {32, 32, 1};
    if (!encode(&g.to, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g.out, d3, s3, b3, CU_TENSOR_MAP_SWIZZLE_128B)) return false;
    const cuuint32_t b2[2] = {32, 32};
    if (g.out_b) {
        const cuuint64_t d2[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
        const cuuint64_t s2[1] = {(cuuint64_t)g.ldob * 2};
        if (!encode(&g.tob, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.out_b, d2, s2, b2, CU_TENSOR_MAP_SWIZZLE_64B))
            return false;
    }
    if (g.out_t) {
        const cuuint64_t d2[2] = {(cuuint64_t)g.M, (cuuint64_t)g.N};
        const cuuint64_t s2[1] = {(cuuint64_t)g.ldt * 2};
        if (!encode(&g.tot, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.out_t, d2, s2, b2, CU_TENSOR_MAP_SWIZZLE_NONE))
            return false;
    }
    return true;
}

static bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool gemm_tma_ok(const TmaGemm& g) {
    if (g.M < 1 || g.N < 1 || g.N > 256 || g.K < 1 || g.nsplit < 1 || !g.out) return false;
    if (!g.a || !g.b || !al16(g.a) || !al16(g.b) || g.lda % 8 || g.ldb % 8 || g.lda < g.K || g.ldb < g.K) return false;
    if (g.nsplit > 1 && (g.epi != EPI_STORE || g.split_stride % 4 || g.split_stride < (long)g.M * g.ldo)) return false;
    if (!al16(g.out) || g.ldo % 4 || g.ldo < g.N) return false;
    if (g.out_b && (!al16(g.out_b) || g.ldob % 8 || g.ldob < g.N)) return false;
    if (g.out_t && (!al16(g.out_t) || g.ldt % 8 || g.ldt < g.M)) return false;
    if ((g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) && (!g.bias || !al16(g.bias))) return false;
    if (g.epi == EPI_GELU_BWD && (!g.aux || !al16(g.aux) || g.ldaux % 4 || g.ldaux < g.N)) return false;
    return true;
}

static int sm_count() {
    static int n[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n[dev] = 148;
    return n[dev];
}

int gemm_tma_nt(int M, int N, int nsplit) {
    if (N <= 64) return 64;
    const long mt = (M + 127) / 128 * (long)nsplit, sms = sm_count();
    if (mt * ((N + 255) / 256) >= sms) return 256;
    if (mt * ((N + 127) / 128) >= sms) return 128;
    return 64;
}

int gemm_tma_split(int M, int K, int max_split) {
    const int mtiles = (M + 127) / 128, nk = (K + 63) / 64;
    const int target = sm_count() / mtiles;
    if (target <= 1 || max_split <= 1) return 1;
    int kcs = (nk + target - 1) / target;
    if (kcs < 4) kcs = 4;
    int ns = (nk + kcs - 1) / kcs;
    if (ns > max_split) {
        kcs = (nk + max_split - 1) / max_split;
        ns = (nk + kcs - 1) / kcs;
    }
    return ns < 1 ? 1 : ns;
}

template <int NT>
static cudaError_t launch_nt(const TmaGemm& g, cudaStream_t st) {
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_gemm_tma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GtCfg<NT>::SMEM);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_tma<NT>, GT_THREADS, GtCfg<NT>::SMEM) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        // two accumulators of NT columns per CTA must fit the SM's 512 TMEM columns
        if (per_sm * GtCfg<NT>::TCOLS > 512) per_sm = 512 / GtCfg<NT>::TCOLS;
    });
    const int units = ((g.M + 127) / 128) * g.ntiles * g.nsplit;
    const int grid = units < per_sm * sm_count() ? units : per_sm * sm_count();
    k_gemm_tma<NT><<<grid, GT_THREADS, GtCfg<NT>::SMEM, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tma(const TmaGemm& g0, cudaStream_t st) {
    if (!gemm_tma_ok(g0)) return cudaErrorInvalidValue;
    TmaGemm g = g0;
    const int nk = (g.K + 63) / 64;
    g.kcs = (nk + g.nsplit - 1) / g.nsplit;
    if ((g.nsplit - 1) * g.kcs >= nk) return cudaErrorInvalidValue;  // a range would be empty
    const int nt = gemm_tma_nt(g.M, g.N, g.nsplit);
    g.ntiles = (g.N + nt - 1) / nt;
    if (!encode_kmajor(&g.ta, g.a, g.M, g.K, g.lda, 128) || !encode_kmajor(&g.tb, g.b, g.N, g.K, g.ldb, nt) ||
        !encode_outputs(g))
        return cudaErrorInvalidValue;
    return nt == 64 ? launch_nt<64>(g, st) : (nt == 128 ? launch_nt<128>(g, st) : launch_nt<256>(g, st));
}

}  // namespace mppi
