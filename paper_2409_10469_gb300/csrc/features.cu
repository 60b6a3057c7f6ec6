// features.cu -- the features kernel and its entry points; the 62 numbers
// (features.cuh) describe the robot, the free box and the task at one control step.
#include <math.h>

#include "features.cuh"
#include "handle.h"
#include "memkind.h"

namespace mppi {

struct FeatArgs {
    const float* X;
    int n, ldx;
    FeatParams p;
    float* F;
};

__global__ void k_features(FeatArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    state_features(a.X + (size_t)i * a.ldx, a.p, a.F + (size_t)i * 62);
}

}  // namespace mppi

using namespace mppi;

// memory of the current device (or managed memory)
static bool fdev(const void* p) { return is_local(p); }

// the handle's device is the current one and no buffer is another GPU's memory
static bool local_call(mppi_handle h, std::initializer_list<const void*> bufs) {
    const int dev = current_device();
    if (dev != h->device) {
        h->err = "the handle's device is not the current device";
        return false;
    }
    if (any_foreign(dev, bufs)) {
        h->err = "a buffer is memory of another GPU";
        return false;
    }
    return true;
}

// what the features take besides the state, for this handle at control index `step`
FeatParams mppi_feature_params(mppi_handle h, uint32_t step) {
    FeatParams p;
    p.nx = h->nx;
    p.goal_x = (float)h->cost_in.goal_xy[0];
    p.goal_y = (float)h->cost_in.goal_xy[1];
    p.box_gx = (float)h->cost_in.box_goal_xy[0];
    p.box_gy = (float)h->cost_in.box_goal_xy[1];
    const double t = (double)step * h->cfg.ctrl_steps * h->cfg.dt;
    const double P = h->cost_in.gait_period;
    p.phase = ((h->cost_in.gait == 1 || h->cost_in.gait == 2) && P > 0) ? (float)(2.0 * M_PI * fmod(t, P) / P) : 0.f;
    return p;
}

// k_features over n device states dX of this handle at control index `step`,
// into device dF [n][62], on stream st
static cudaError_t launch_features(mppi_handle h, const float* dX, int n, uint32_t step, float* dF, cudaStream_t st) {
    FeatArgs a;
    a.X = dX;
    a.n = n;
    a.ldx = h->nx;
    a.p = mppi_feature_params(h, step);
    a.F = dF;
    k_features<<<(n + 127) / 128, 128, 0, st>>>(a);
    h->launches++;
    return cudaGetLastError();
}

extern "C" mppi_status mppi_features(mppi_handle h, const float* X, int n, uint32_t step, float* F) {
    if (!h || !X || !F || n < 1) return MPPI_ERR_ARG;
    if (!local_call(h, {X, F})) return MPPI_ERR_ARG;
    const int nx = h->nx;
    cudaStream_t st = h->stream;
    float *dX = nullptr, *dF = nullptr;
    const bool xdev = fdev(X), fdv = fdev(F);
    if (!xdev && cudaMalloc((void**)&dX, (size_t)n * nx * 4) != cudaSuccess) return MPPI_ERR_OOM;
    if (!fdv && cudaMalloc((void**)&dF, (size_t)n * 62 * 4) != cudaSuccess) {
        if (dX) cudaFree(dX);
        return MPPI_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    if (!xdev) e = cudaMemcpyAsync(dX, X, (size_t)n * nx * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_features(h, xdev ? X : dX, n, step, fdv ? F : dF, st);
    if (e == cudaSuccess && !fdv) e = cudaMemcpyAsync(F, dF, (size_t)n * 62 * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && (!fdv || !xdev)) e = cudaStreamSynchronize(st);
    if (dX) cudaFree(dX);
    if (dF) cudaFree(dF);
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

extern "C" mppi_status mppi_set_proposal(mppi_handle h, const float* mu_prop) {
    if (!h) return MPPI_ERR_ARG;
    if (!mu_prop) {
        h->has_prop = 0;
        return MPPI_OK;
    }
    if (h->cfg.n_prop < 1) {
        h->err = "the handle was created with n_prop = 0";
        return MPPI_ERR_ARG;
    }
    if (!local_call(h, {mu_prop})) return MPPI_ERR_ARG;
    const cudaMemcpyKind k = fdev(mu_prop) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(h->d_mu_prop, mu_prop, D * sizeof(float), k, h->stream) != cudaSuccess) return MPPI_ERR_CUDA;
    if (k == cudaMemcpyHostToDevice && cudaStreamSynchronize(h->stream) != cudaSuccess) return MPPI_ERR_CUDA;
    h->has_prop = 1;
    return MPPI_OK;
}
