// features.cu -- input features of the proposal network: 62 numbers describing
// the robot, the free box and the task at one control step (model spec).
//   0      trunk height
//   1-4    trunk quaternion (w, x, y, z), sign chosen so that w >= 0
//   5-16   joint angles
//   17-19  trunk angular velocity (body)      20-22 linear velocity (body)
//   23-34  joint rates x 0.1
//   35-36  box xy - trunk xy                  37    box height
//   38-41  box quaternion (w >= 0)            42-44 box angular velocity (body)
//   45-47  box linear velocity (body)         48-49 box goal xy - box xy
//   50-51  trunk goal xy - trunk xy           52-53 sin, cos of the gait phase
//   54-56  gravity direction in the trunk frame (R^T e_z)
//   57-58  box heading (first column of the box rotation, xy)
//   59     |box goal - box| (xy)              60    |box - trunk| (xy)
//   61     1
// Box entries are zero for a robot without a box.
#include <math.h>

#include "handle.h"

namespace mppi {

struct FeatArgs {
    const float* X;
    int n, nx, ldx;
    float goal_x, goal_y, box_gx, box_gy, phase;  // phase = 2 pi t / period (0 without a gait)
    float* F;
};

__global__ void k_features(FeatArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float* x = a.X + (size_t)i * a.ldx;
    float* f = a.F + (size_t)i * 62;
    f[0] = x[2];
    const float sq = x[3] < 0.f ? -1.f : 1.f;
    for (int j = 0; j < 4; j++) f[1 + j] = sq * x[3 + j];
    for (int j = 0; j < 12; j++) f[5 + j] = x[7 + j];
    for (int j = 0; j < 6; j++) f[17 + j] = x[19 + j];
    for (int j = 0; j < 12; j++) f[23 + j] = 0.1f * x[25 + j];
    const bool box = a.nx >= NX_BOX;
    const float bx = box ? x[37] : 0.f, by = box ? x[38] : 0.f;
    f[35] = box ? bx - x[0] : 0.f;
    f[36] = box ? by - x[1] : 0.f;
    f[37] = box ? x[39] : 0.f;
    const float sb = (box && x[40] < 0.f) ? -1.f : 1.f;
    for (int j = 0; j < 4; j++) f[38 + j] = box ? sb * x[40 + j] : 0.f;
    for (int j = 0; j < 6; j++) f[42 + j] = box ? x[44 + j] : 0.f;
    f[48] = box ? a.box_gx - bx : 0.f;
    f[49] = box ? a.box_gy - by : 0.f;
    f[50] = a.goal_x - x[0];
    f[51] = a.goal_y - x[1];
    float sp, cp;
    sincosf(a.phase, &sp, &cp);
    f[52] = sp;
    f[53] = cp;
    const float w = x[3], qx = x[4], qy = x[5], qz = x[6];
    f[54] = 2.f * (qx * qz - w * qy);
    f[55] = 2.f * (qy * qz + w * qx);
    f[56] = 1.f - 2.f * (qx * qx + qy * qy);
    if (box) {
        const float bw = x[40], bqx = x[41], bqy = x[42], bqz = x[43];
        f[57] = 1.f - 2.f * (bqy * bqy + bqz * bqz);
        f[58] = 2.f * (bqx * bqy + bw * bqz);
    } else {
        f[57] = 0.f;
        f[58] = 0.f;
    }
    f[59] = box ? sqrtf(f[48] * f[48] + f[49] * f[49]) : 0.f;
    f[60] = box ? sqrtf(f[35] * f[35] + f[36] * f[36]) : 0.f;
    f[61] = 1.f;
}

}  // namespace mppi

using namespace mppi;

static bool fdev(const void* p) {
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" mppi_status mppi_features(mppi_handle h, const float* X, int n, uint32_t step, float* F) {
    if (!h || !X || !F || n < 1) return MPPI_ERR_ARG;
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
    FeatArgs a;
    a.X = xdev ? X : dX;
    a.n = n;
    a.nx = nx;
    a.ldx = nx;
    a.goal_x = (float)h->cost_in.goal_xy[0];
    a.goal_y = (float)h->cost_in.goal_xy[1];
    a.box_gx = (float)h->cost_in.box_goal_xy[0];
    a.box_gy = (float)h->cost_in.box_goal_xy[1];
    const double t = (double)step * h->cfg.ctrl_steps * h->cfg.dt;
    const double P = h->cost_in.gait_period;
    a.phase = ((h->cost_in.gait == 1 || h->cost_in.gait == 2) && P > 0) ? (float)(2.0 * M_PI * fmod(t, P) / P) : 0.f;
    a.F = fdv ? F : dF;
    if (e == cudaSuccess) {
        k_features<<<(n + 127) / 128, 128, 0, st>>>(a);
        e = cudaGetLastError();
        h->launches++;
    }
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
    const cudaMemcpyKind k = fdev(mu_prop) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(h->d_mu_prop, mu_prop, D * sizeof(float), k, h->stream) != cudaSuccess) return MPPI_ERR_CUDA;
    if (k == cudaMemcpyHostToDevice && cudaStreamSynchronize(h->stream) != cudaSuccess) return MPPI_ERR_CUDA;
    h->has_prop = 1;
    return MPPI_OK;
}
