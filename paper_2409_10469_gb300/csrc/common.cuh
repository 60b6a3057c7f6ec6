// common.cuh -- device-side model, cost and small spatial-algebra helpers for
// the sm_103a MPPI kernels (arXiv 2409.10469; simulator per the model spec that
// replaces the paper's MuJoCo rollouts, Sec. III-A).
//
// Spatial vectors are [angular; linear] in body coordinates (Featherstone).
// A spatial inertia is stored as the symmetric 6x6 [[A, B], [B^T, C]] with A, C
// symmetric 3x3 and B a general 3x3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mppi {

constexpr int NJ = 12;
constexpr int NKNOT = 4;
constexpr int D = NKNOT * NJ;
constexpr int NX_ROBOT = 37;
constexpr int NX_BOX = 50;
constexpr int MAX_SBOX = 4;

struct Sym6 {
    float A[3][3];  // symmetric
    float B[3][3];
    float C[3][3];  // symmetric
};

// All derived, FP32 model constants (computed on the host from mppi_model_t).
struct DevModel {
    float tr_Ic[3], tr_m;             // trunk: principal inertia about its centre, mass
    Sym6 I_hip, I_thigh, I_calf;      // leg bodies: spatial inertia about the joint origin
    float r_hip[4][3];                // abduction joint in the trunk frame
    float r_thigh[4][3];              // flexion joint in the hip frame
    float r_knee[3];                  // knee in the thigh frame
    float foot[3], foot_r;            // foot sphere centre in the calf frame, radius
    int n_tsph;
    float tsph_x[4], tsph_r;          // trunk spheres on the trunk x axis
    float gz;                         // gravity (world z component, negative)
    float kp, kd, arm0;
    float kc, cc, mu, eps2;           // contact stiffness, damping, friction, eps_v^2
    int terrain;                      // 0 plane, 1 heightfield
    int hf_nx, hf_ny;
    float hf_cell, hf_inv_cell, hf_x0, hf_y0;
    const float* hf;                  // device heights [ny][nx]
    int n_sbox;
    float sb_lo[MAX_SBOX][3], sb_hi[MAX_SBOX][3];
    int has_box;
    float box_m, box_inv_m, box_half[3], box_Ic[3], box_inv_Ic[3], box_cr;
    int nx;
};

struct DevCost {
    float w_z, z_ref, w_o, w_v, v_ref, w_p, goal_x, goal_y, w_u, w_box, box_gx, box_gy;
    int gait;
    float two_pi_over_period, hip_amp, knee_amp;
    float stand[3];
    float w_term;
};

// ---------------------------------------------------------------- float3 ops
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 ld3(const float* p) { return f3(p[0], p[1], p[2]); }

// Coordinate rotations (parent -> child coordinates, E) of a frame turned by +q
// about x or y, with (c, s) = (cos q, sin q), and their transposes.
__device__ __forceinline__ float3 Ex(float c, float s, float3 v) { return f3(v.x, c * v.y + s * v.z, c * v.z - s * v.y); }
__device__ __forceinline__ float3 ExT(float c, float s, float3 v) { return f3(v.x, c * v.y - s * v.z, s * v.y + c * v.z); }
__device__ __forceinline__ float3 Ey(float c, float s, float3 v) { return f3(c * v.x - s * v.z, v.y, s * v.x + c * v.z); }
__device__ __forceinline__ float3 EyT(float c, float s, float3 v) { return f3(c * v.x + s * v.z, v.y, c * v.z - s * v.x); }

template <int AX> __device__ __forceinline__ float3 Erot(float c, float s, float3 v) {
    return AX == 0 ? Ex(c, s, v) : Ey(c, s, v);
}
template <int AX> __device__ __forceinline__ float3 ErotT(float c, float s, float3 v) {
    return AX == 0 ? ExT(c, s, v) : EyT(c, s, v);
}

// M <- R M R^T with R = E^T (child -> parent rotation), for a general 3x3 M.
template <int AX> __device__ __forceinline__ void rot3(float M[3][3], float c, float s) {
    // rows then columns; AX 0 mixes (1, 2), AX 1 mixes (0, 2)
    constexpr int i0 = AX == 0 ? 1 : 0;
    constexpr int i1 = 2;
    // R for AX 0: row1 = c e1 - s e2, row2 = s e1 + c e2 ; AX 1: row0 = c e0 + s e2, row2 = -s e0 + c e2
    const float sg = AX == 0 ? -1.f : 1.f;  // sign of the s term in the first mixed row
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float a = M[i0][j], b = M[i1][j];
        M[i0][j] = c * a + sg * s * b;
        M[i1][j] = c * b - sg * s * a;
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float a = M[i][i0], b = M[i][i1];
        M[i][i0] = c * a + sg * s * b;
        M[i][i1] = c * b - sg * s * a;
    }
}

// Congruence of a spatial inertia into the parent frame: X^T M X with
// X = rot(E) xlt(r) (joint rotation about AX, then the joint origin r):
//   rotate every block by E^T, then
//   A'' = A' - (P + P^T) - Q,  B'' = B' + r x C',  C'' = C',
//   P = B' [r x],  Q = [r x] C' [r x].
template <int AX>
__device__ __forceinline__ void congruence(Sym6& M, float c, float s, float3 r) {
    rot3<AX>(M.A, c, s);
    rot3<AX>(M.B, c, s);
    rot3<AX>(M.C, c, s);
    float P[3][3], T[3][3], Q[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        P[i][0] = M.B[i][1] * r.z - M.B[i][2] * r.y;
        P[i][1] = M.B[i][2] * r.x - M.B[i][0] * r.z;
        P[i][2] = M.B[i][0] * r.y - M.B[i][1] * r.x;
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        T[0][j] = r.y * M.C[2][j] - r.z * M.C[1][j];
        T[1][j] = r.z * M.C[0][j] - r.x * M.C[2][j];
        T[2][j] = r.x * M.C[1][j] - r.y * M.C[0][j];
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Q[i][0] = T[i][1] * r.z - T[i][2] * r.y;
        Q[i][1] = T[i][2] * r.x - T[i][0] * r.z;
        Q[i][2] = T[i][0] * r.y - T[i][1] * r.x;
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            M.A[i][j] = M.A[i][j] - (P[i][j] + P[j][i]) - Q[i][j];
            M.B[i][j] = M.B[i][j] + T[i][j];
        }
}

__device__ __forceinline__ void sym6_add(Sym6& a, const Sym6& b) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            a.A[i][j] += b.A[i][j];
            a.B[i][j] += b.B[i][j];
            a.C[i][j] += b.C[i][j];
        }
}

// I [w; v]
__device__ __forceinline__ void sym6_mv(const Sym6& M, float3 w, float3 v, float3& ha, float3& hl) {
    ha = f3(M.A[0][0] * w.x + M.A[0][1] * w.y + M.A[0][2] * w.z + M.B[0][0] * v.x + M.B[0][1] * v.y + M.B[0][2] * v.z,
            M.A[1][0] * w.x + M.A[1][1] * w.y + M.A[1][2] * w.z + M.B[1][0] * v.x + M.B[1][1] * v.y + M.B[1][2] * v.z,
            M.A[2][0] * w.x + M.A[2][1] * w.y + M.A[2][2] * w.z + M.B[2][0] * v.x + M.B[2][1] * v.y + M.B[2][2] * v.z);
    hl = f3(M.B[0][0] * w.x + M.B[1][0] * w.y + M.B[2][0] * w.z + M.C[0][0] * v.x + M.C[0][1] * v.y + M.C[0][2] * v.z,
            M.B[0][1] * w.x + M.B[1][1] * w.y + M.B[2][1] * w.z + M.C[1][0] * v.x + M.C[1][1] * v.y + M.C[1][2] * v.z,
            M.B[0][2] * w.x + M.B[1][2] * w.y + M.B[2][2] * w.z + M.C[2][0] * v.x + M.C[2][1] * v.y + M.C[2][2] * v.z);
}

// rotation matrix (body -> world) of a unit quaternion (w, x, y, z)
__device__ __forceinline__ void quat_R(const float q[4], float R[3][3]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z);       R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);       R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);       R[2][1] = 2.f * (y * z + w * x);       R[2][2] = 1.f - 2.f * (x * x + y * y);
}
__device__ __forceinline__ float3 mulR(const float R[3][3], float3 v) {
    return f3(R[0][0] * v.x + R[0][1] * v.y + R[0][2] * v.z, R[1][0] * v.x + R[1][1] * v.y + R[1][2] * v.z,
              R[2][0] * v.x + R[2][1] * v.y + R[2][2] * v.z);
}
__device__ __forceinline__ float3 mulRT(const float R[3][3], float3 v) {
    return f3(R[0][0] * v.x + R[1][0] * v.y + R[2][0] * v.z, R[0][1] * v.x + R[1][1] * v.y + R[2][1] * v.z,
              R[0][2] * v.x + R[1][2] * v.y + R[2][2] * v.z);
}

// quaternion q <- normalise(q (x) exp(w h)), w in body coordinates
__device__ __forceinline__ void quat_integrate(float q[4], float3 w, float h) {
    float wn = sqrtf(dot3(w, w));
    float th = wn * h;
    float sh, ch;
    sincosf(0.5f * th, &sh, &ch);
    float sk = (th > 1e-4f) ? sh / wn : 0.5f * h * (1.f - th * th * (1.f / 24.f));
    float d0 = ch, d1 = sk * w.x, d2 = sk * w.y, d3 = sk * w.z;
    float r0 = q[0] * d0 - q[1] * d1 - q[2] * d2 - q[3] * d3;
    float r1 = q[0] * d1 + q[1] * d0 + q[2] * d3 - q[3] * d2;
    float r2 = q[0] * d2 - q[1] * d3 + q[2] * d0 + q[3] * d1;
    float r3 = q[0] * d3 + q[1] * d2 - q[2] * d1 + q[3] * d0;
    float inv = 1.f / sqrtf(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    q[0] = r0 * inv; q[1] = r1 * inv; q[2] = r2 * inv; q[3] = r3 * inv;
}

}  // namespace mppi
