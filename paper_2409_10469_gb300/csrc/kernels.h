// kernels.h -- internal launch interface between the C-ABI layer (api.cu) and
// the kernels (sample.cu, rollout.cu, update.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace mppi {

struct SampleArgs {
    const float* mu;       // [48] device
    const float* mu_prop;  // [48] device or null
    float* U;              // [K][Dp] device
    float sigma[D];        // per knot and joint (DIRECT: sigma[i] for joint i)
    float q_lo[3], q_hi[3];
    uint32_t key0, key1, step, inst;
    int K, n_prop;
    int Dp;                // parameters per sample: 48, or 12 H (DIRECT)
    int interp;            // MPPI_INTERP_*
    uint32_t g_magic;      // floor(2^32 / (Dp / 4)), set by launch_sample
};

struct RolloutArgs {
    DevModel model;
    DevCost cost;
    const float* x0;       // [nx] or [n][nx] device
    int x0_per_sample;
    const float* U;        // [n][Dp] device
    float* L;              // [n] device
    float* traj;           // [n][H+1][nx] device or null
    int n, H, n_sub;
    int Dp, interp;        // parameters per sample, MPPI_INTERP_*
    const float4* Bt;      // [H] knot weights of each dt step (knot representations)
    float h, dt, inv_Hm1, t0;  // t0: gait time of step 0 (reduced modulo the gait period)
    float arm;             // implicit-PD armature h (kd + h kp) + a0
    // in-kernel sampling (the control step, knot representations): each lane draws
    // its leg's 12 knots exactly as k_sample would and writes them to U_out
    int sample;
    int k_off;             // global index of sample 0 of this launch (a shard of a K-sample step)
    const float* mu;       // [48] nominal
    const float* mu_prop;  // [48] proposal mean or null
    int K_all, n_prop;     // the sample set's size and its proposal share
    float sigma[D];
    float q_lo[3], q_hi[3];
    uint32_t key0, key1, step, inst;
    float* U_out;          // [n][48]
    // fused update (the control step, knot representations): each CTA folds its
    // rollouts into FP64 partial sums around its own cost minimum, the last CTA
    // to finish combines them (Eq. 1, Eq. 2), applies and shifts; these are the
    // outputs and scratch of UpdateArgs, with part sized FUSE_W per CTA
    int fuse;
    double inv_lambda;     // 1 / lambda (FP64: the weights' exponent is formed in FP64)
    int ctrl_steps;
    float* mu_w;           // [48] the nominal (== mu), overwritten by the shifted nominal
    float* mu_upd;         // [48]
    float* u0;             // [12]
    int* status;
    double* wsum;
    double* part;          // [grid][FUSE_W] (used as float pairs)
    unsigned* counter;     // 0 between launches
    // the outputs again in pinned, device-mapped host memory (the handle's
    // mailbox), for callers that want them on the host, or null: u0 [12],
    // mu' [48], status
    float* u0_host;
    float* mu_host;
    int* status_host;
};

constexpr int FUSE_W = D + 2;  // per-CTA partial: 48 weighted sums, the weight sum, the CTA's cost minimum
constexpr int FUSE_MAX_CTAS = 1024;  // grids up to this size fuse the update (its factors sit in shared memory)

struct UpdateArgs {
    const float* L;        // [n]
    const float* U;        // [n][Dp]
    float* mu;             // [Dp] in: the previous mean (kept when no cost is finite); out: shifted nominal
    float* mu_upd;         // [Dp] updated mean before the shift (required when Dp > 48)
    float* u0;             // [12]
    int* status;           // 0 ok, 4 all costs non-finite
    double* wsum;          // normaliser (FP64) of the last update, optional
    double* part;          // scratch: per-chunk partial sums, weight sum, cost minimum ([grid][50] for
                           // knots, [chunks][Dp + 2] for direct targets)
    unsigned* counter;     // scratch: CTAs finished (0 between launches)
    int n, H, ctrl_steps;
    double inv_lambda;     // 1 / lambda (FP64: the weights' exponent is formed in FP64)
    int Dp, interp;        // parameters per sample, MPPI_INTERP_*
    double* partial_out;   // launch_update_partial: [50] L_min, Z, S[48] of these samples
};

// Eq. 2's combined sums of a sharded step (Z, S[48], relative to the global
// L_min) -> mu' = S / Z, u0, the shifted nominal and the status (one CTA)
struct FinalizeArgs {
    const double* sums;    // [49] Z, S[48] (device)
    float* mu;             // [48] in: the nominal (kept when Z is not positive and finite); out: shifted
    float* mu_upd;         // [48]
    float* u0;             // [12]
    int* status;
    int H, ctrl_steps, interp;
};

constexpr int UPDATE_MAX_CTAS = 128;
int update_grid(int n);
// parameter tiles of 48 for Dp parameters per sample, the update scratch's
// doubles and its counters
constexpr int update_tiles(int Dp) { return (Dp + D - 1) / D; }
constexpr size_t update_part_doubles(int Dp) { return (size_t)UPDATE_MAX_CTAS * update_tiles(Dp) * (D + 2); }
constexpr int update_counters(int Dp) { return 1 + update_tiles(Dp); }
// direct targets (Dp = 12 H): the most sample chunks an update of Dp parameters
// per sample uses, and its scratch in doubles (any n: the chunk count is capped)
int update_direct_chunks_cap(int Dp);
size_t update_direct_part_doubles(int Dp);

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st);
// the noise self-test's tables (2^24 entries each)
cudaError_t launch_noise_tables(float* radius, float* cosv, float* sinv, cudaStream_t st);
cudaError_t launch_rollout(const RolloutArgs& a, int block, cudaStream_t st);
// CTAs of a rollout launch of n samples at this block size
inline int rollout_grid(int n, int block) { return (int)((4L * n + block - 1) / block); }
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st);
// the partial sums of the knot representations' update over a.n samples: the
// samples' finite-cost minimum m, Z = sum exp(-(L - m) / lambda) and
// S = sum exp(-(L - m) / lambda) U, into a.partial_out (no mean, no shift)
cudaError_t launch_update_partial(const UpdateArgs& a, cudaStream_t st);
cudaError_t launch_update_finalize(const FinalizeArgs& a, cudaStream_t st);

}  // namespace mppi
