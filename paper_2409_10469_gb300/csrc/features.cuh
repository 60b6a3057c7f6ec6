// features.cuh -- input features of the proposal network: 62 numbers describing
// the robot, the free box and the task at one control step (model spec), as
// one thread computes them for one state.  Used by the features kernel and by
// the fused small-batch forward of the proposal network.
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
#pragma once
#include <math.h>

#include "common.cuh"

namespace mppi {

// what the features take besides the state
struct FeatParams {
    int nx;                                       // state length (NX_BOX or more: a box is present)
    float goal_x, goal_y, box_gx, box_gy, phase;  // phase = 2 pi t / period (0 without a gait)
};

// the 62 features of state x into f (global or shared memory)
__device__ __forceinline__ void state_features(const float* x, const FeatParams& a, float* f) {
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
    const float dbx = f[48], dby = f[49], dtx = f[35], dty = f[36];
    f[59] = box ? sqrtf(dbx * dbx + dby * dby) : 0.f;
    f[60] = box ? sqrtf(dtx * dtx + dty * dty) : 0.f;
    f[61] = 1.f;
}

}  // namespace mppi
