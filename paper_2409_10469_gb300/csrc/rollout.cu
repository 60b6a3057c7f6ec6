// rollout.cu -- K2: MPPI rollouts of one instance on sm_103a CUDA cores (FP32).
//
// arXiv 2409.10469, Alg. 1 inner loop: every sample's knot vector is turned into
// joint targets by the cubic spline (Sec. III-B), tracked by PD (Sec. IV-A) and
// simulated for T steps while L_walk (Sec. IV-B) and L_box (Sec. IV-D) accumulate.
// The per-lane arithmetic lives in rollout.cuh; this kernel maps 4 lanes to a
// rollout (8 rollouts per warp) over the n samples of one controller.
#include "kernels.h"
#include "noise.cuh"
#include "rollout.cuh"

namespace mppi {

template <int TERR, bool BOX, bool DIRECT>
__global__ void __launch_bounds__(256, 1) k_rollout(RolloutArgs a) {
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
        // fmaf perturbation, clamp), so the knots are bit-identical to it
        const int kp0 = a.K_all - (a.mu_prop ? a.n_prop : 0);
        const bool prop = a.mu_prop && kk >= kp0;
        const float* ctr = prop ? a.mu_prop : a.mu;
        const bool nominal = (kk == 0) || (prop && kk == kp0);
#pragma unroll
        for (int j = 0; j < NKNOT; j++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int d = j * NJ + 3 * leg + i;
                const float eps = nominal ? 0.f : normal_at(a.key0, a.key1, a.step, a.inst, (uint32_t)kk, d);
                float c = __ldg(ctr + d);
                if (prop && !(fabsf(c) <= 3.402823466e38f)) c = __ldg(a.mu + d);  // non-finite proposal: plain mean
                const float v = fminf(fmaxf(__fmaf_rn(a.sigma[d], eps, c), a.q_lo[i]), a.q_hi[i]);
                Uk[j][i] = v;
                if (valid) a.U_out[(size_t)kk * D + d] = v;
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
