// gemm.h -- the TMA-fed BF16 tcgen05 GEMM D = A B^T (gemm.cu) as the proposal
// network (mlp.cu) and the raw GEMM entry point use it, plus the epilogue
// functions both tensor-core kernels share.
#pragma once
#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched from the driver at run time
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace mppi {

enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
// d/dz of z Phi(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// D[M][N] = A[M][K] B[N][K]^T with A and B BF16, K contiguous (rows lda and ldb
// elements apart), N <= 256, fed to the kernel by TMA.  Output tiles are 128
// rows x NT columns, NT = 256, 128 or 64: the widest whose tile count still
// fills the SMs (N <= 64: 64).  Epilogue on the FP32 sum d:
//   EPI_STORE       out = d
//   EPI_BIAS        out = d + bias[n]
//   EPI_BIAS_GELU   out = d + bias[n], out_b = out_t^T = bf16(gelu(out))
//   EPI_GELU_BWD    out = d * gelu'(aux[m][n]), out_b = out_t^T = bf16(out)
// out_b (row-major) and out_t (transposed: out_t[n * ldt + m]) are optional.
// Split-K: K is cut into nsplit ranges of whole 64-wide chunks and range sp
// writes its partial sum (EPI_STORE only) to out + sp * split_stride.
// Requirements (checked by gemm_tma_ok): a, b 16-byte aligned, lda and ldb
// multiples of 8; out 16-byte aligned, ldo % 4 == 0, split_stride % 4 == 0;
// out_b 16-byte aligned, ldob % 8 == 0; out_t 16-byte aligned, ldt % 8 == 0;
// aux 16-byte aligned, ldaux % 4 == 0.
struct TmaGemm {
    // tensor maps, encoded by launch_gemm_tma from the pointers below
    CUtensorMap ta, tb;    // A boxes 128 x 64, B boxes NT x 64 (128-byte swizzle)
    CUtensorMap to, tob;   // out [nsplit][M][ldo] FP32 and out_b [M][ldob] BF16
    CUtensorMap tot;       // out_t [N][ldt] BF16
    const __nv_bfloat16* a;
    long lda;
    const __nv_bfloat16* b;
    long ldb;
    int M, N, K;
    int nsplit;
    int kcs;               // chunks of 64 per range (set by launch_gemm_tma: ceil(chunks / nsplit))
    int ntiles;            // column tiles of NT (set by launch_gemm_tma)
    long split_stride;
    int epi;
    const float* bias;
    const float* aux;
    long ldaux;
    float* out;
    long ldo;
    __nv_bfloat16* out_b;
    long ldob;
    __nv_bfloat16* out_t;
    long ldt;
    int* err;              // set to 1 when a wait runs out
    uint32_t wait_limit;   // mbarrier polls before giving up (0 = default)
    int withhold_commit;   // self-test: never signal MMA completion, so the waits run out
};

// the operands' and the epilogue's layout requirements hold
bool gemm_tma_ok(const TmaGemm& g);
// split count for an M x K product so that the work units fill the SMs
// (at least 4 chunks of 64 per range, at most max_split ranges, none empty)
int gemm_tma_split(int M, int K, int max_split);
// tile width launch_gemm_tma uses for an M x N product cut into nsplit K ranges
int gemm_tma_nt(int M, int N, int nsplit);
cudaError_t launch_gemm_tma(const TmaGemm& g, cudaStream_t st);

}  // namespace mppi
