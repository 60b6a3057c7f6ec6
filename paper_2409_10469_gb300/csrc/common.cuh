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
// control representations (the ABI's MPPI_INTERP_* values)
constexpr int INTERP_CUBIC = 0, INTERP_ZERO = 1, INTERP_LINEAR = 2, INTERP_DIRECT = 3;

// Symmetric 6x6 [[A, B], [B^T, C]]: A and C by their 6 unique entries
// (order 00 01 02 11 12 22), B in full.
struct Sym6 {
    float A[6];
    float B[3][3];
    float C[6];
};

__host__ __device__ __forceinline__ constexpr int sidx(int i, int j) {
    return i <= j ? (i * (5 - i)) / 2 + j : (j * (5 - j)) / 2 + i;
}

// Spatial inertia of a body whose centre of mass lies on its frame's z axis at
// cz and whose rotational inertia is diagonal there (the hip sphere, the thigh
// and calf rods): about the frame origin A = diag(ax, ay, az) (parallel axis
// included), B = m [c x], C = m 1.
struct BodyI {
    float ax, ay, az, m, mcz;
};

// All derived, FP32 model constants (computed on the host from mppi_model_t).
struct DevModel {
    float tr_Ic[3], tr_m;             // trunk: principal inertia about its centre, mass
    BodyI I_hip, I_thigh, I_calf;     // leg bodies: spatial inertia about the joint origin
    Sym6 Ia_calf;                     // calf articulated inertia after its joint's projection
    float calf_D_inv;                 // 1 / (S^T I_calf S + armature) (the calf's D is constant)
    float hip_x, hip_y, hip_z;        // abduction joint at (+-hip_x, +-hip_y, hip_z) in the trunk frame
    float thigh_y;                    // flexion joint at (0, +-thigh_y, 0) in the hip frame
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
    float sbox[MAX_SBOX * 6];         // [n_sbox][6]: lo xyz, hi xyz, by value (kernel parameters)
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
    float quarter_period, raibert_k, inv_raibert_len;  // gait 2: T_stance / 2, velocity gain, 1 / leg length
    int z_rel;                                          // height reference from the ground under the trunk
};

// shifted(mu) knot j, joint i for the knot representations: the representation's
// interpolant of mu (4 x 12 knots) at tau_j + ctrl / (H - 1), held at tau = 1.
// Cubic: the Lagrange basis; zeroth order / linear: the knot interval at
// 3 tau = j + 3 ctrl / (H - 1), whose integer part and fraction come from
// integer arithmetic.
__device__ __forceinline__ float shifted_knot(const float* mu, int interp, int H, int ctrl, int j, int i) {
    if (interp == INTERP_CUBIC) {
        const float delta = H > 1 ? (float)ctrl / (float)(H - 1) : 0.f;
        const float tau = fminf((float)j * (1.f / 3.f) + delta, 1.f);
        const float d0 = tau, d1 = tau - (1.f / 3.f), d2 = tau - (2.f / 3.f), d3 = tau - 1.f;
        const float B0 = d1 * d2 * d3 * -4.5f, B1 = d0 * d2 * d3 * 13.5f;
        const float B2 = d0 * d1 * d3 * -13.5f, B3 = d0 * d1 * d2 * 4.5f;
        return B0 * mu[i] + B1 * mu[NJ + i] + B2 * mu[2 * NJ + i] + B3 * mu[3 * NJ + i];
    }
    const int den = H > 1 ? H - 1 : 1, num = H > 1 ? 3 * ctrl : 0;
    int jj = j + num / den;
    float f = (float)(num % den) / (float)den;
    if (jj >= 3) {
        jj = 3;
        f = 0.f;
    }
    if (interp == INTERP_ZERO || jj == 3) return mu[jj * NJ + i];
    return (1.f - f) * mu[jj * NJ + i] + f * mu[(jj + 1) * NJ + i];
}

// q = S / Z for float-float S and Z > 0, rounded to FP32: the FP32 quotient of
// the high parts, then one correction from the exact remainder S - q1 Z
// (TwoProd by FMA) over Z's high part
__device__ __forceinline__ float ff_div(float2 S, float2 Z) {
    const float q1 = __fdiv_rn(S.x, Z.x);
    const float ph = __fmul_rn(q1, Z.x), pl = __fmaf_rn(q1, Z.x, -ph);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(S.x, ph), pl), __fmaf_rn(-q1, Z.y, S.y));
    return __fadd_rn(q1, __fdiv_rn(r, Z.x));
}

// Count this CTA in on a global counter after its global writes; returns, to
// every thread, whether this CTA brought the count to `total` (it is the last
// of the CTAs counted), in which case the counted CTAs' writes are visible to
// all its threads.  The barrier gathers the CTA's writes under thread 0, whose
// one atomic add with acquire-release semantics at GPU scope publishes them
// (release is cumulative) and, in the last CTA, acquires the others'; the
// second barrier hands that on to the CTA's other threads.  `flag` is a shared
// int.  No thread waits on another CTA.
__device__ __forceinline__ bool cta_count_in(unsigned* counter, unsigned inc, unsigned total, int& flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(prev) : "l"(counter), "r"(inc) : "memory");
        flag = prev + inc == total;
    }
    __syncthreads();
    return flag != 0;
}

// MUFU reciprocal and reciprocal square root with subnormals flushed to zero:
// one instruction each, no subnormal-handling branch (the arguments here --
// pivots, determinants, norms plus a positive floor -- are never subnormal)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

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

// c + a x b with every component one fused chain
__device__ __forceinline__ float3 cross_acc(float3 a, float3 b, float3 c) {
    return f3(fmaf(a.y, b.z, fmaf(-a.z, b.y, c.x)), fmaf(a.z, b.x, fmaf(-a.x, b.z, c.y)),
              fmaf(a.x, b.y, fmaf(-a.y, b.x, c.z)));
}
// c + a x (0, r, 0) and c + a x (0, 0, r), the structurally-zero products left out
// (IEEE arithmetic does not let the compiler drop x * 0 by itself)
__device__ __forceinline__ float3 cross_y_acc(float3 a, float r, float3 c) {
    return f3(fmaf(-a.z, r, c.x), c.y, fmaf(a.x, r, c.z));
}
__device__ __forceinline__ float3 cross_z_acc(float3 a, float r, float3 c) {
    return f3(fmaf(a.y, r, c.x), fmaf(-a.x, r, c.y), c.z);
}

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

// ---------------------------------------------------------------- congruence
// R = E^T (child -> parent) for a joint about AX mixes indices p, q and keeps o:
// AX 0 (x): (p, q) = (1, 2), R = [1 0 0; 0 c -s; 0 s c] -> sigma = -1
// AX 1 (y): (p, q) = (0, 2), R = [c 0 s; 0 1 0; -s 0 c] -> sigma = +1
template <int AX> struct RotIdx {
    static constexpr int o = AX == 0 ? 0 : 1, p = AX == 0 ? 1 : 0, q = 2;
    static constexpr float sg = AX == 0 ? -1.f : 1.f;
};

// S <- R S R^T (+ diag(d) when ADD) for a symmetric 3x3 in unique storage.  The
// rotated diagonal entries take d as the seed of their FMA chains, so only the
// entry on the joint axis pays an addition.
template <int AX, bool ADD>
__device__ __forceinline__ void rot_sym(float S[6], float c, float s, float3 d) {
    using I = RotIdx<AX>;
    const float dg[3] = {d.x, d.y, d.z};
    const float cs = I::sg * c * s, cc = c * c, ss = s * s;
    const float Sop = S[sidx(I::o, I::p)], Soq = S[sidx(I::o, I::q)];
    const float Spp = S[sidx(I::p, I::p)], Sqq = S[sidx(I::q, I::q)], Spq = S[sidx(I::p, I::q)];
    S[sidx(I::o, I::p)] = fmaf(c, Sop, I::sg * s * Soq);
    S[sidx(I::o, I::q)] = fmaf(c, Soq, -I::sg * s * Sop);
    const float t2 = 2.f * cs;
    S[sidx(I::p, I::p)] = fmaf(cc, Spp, fmaf(ss, Sqq, fmaf(t2, Spq, ADD ? dg[I::p] : 0.f)));
    S[sidx(I::q, I::q)] = fmaf(cc, Sqq, fmaf(ss, Spp, fmaf(-t2, Spq, ADD ? dg[I::q] : 0.f)));
    S[sidx(I::p, I::q)] = fmaf(cc - ss, Spq, cs * (Sqq - Spp));
    if (ADD) S[sidx(I::o, I::o)] += dg[I::o];
}

// B <- R B R^T for a general 3x3
template <int AX>
__device__ __forceinline__ void rot_gen(float B[3][3], float c, float s) {
    using I = RotIdx<AX>;
    const float ss_ = I::sg * s;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float a = B[I::p][j], b = B[I::q][j];
        B[I::p][j] = fmaf(c, a, ss_ * b);
        B[I::q][j] = fmaf(c, b, -ss_ * a);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float a = B[i][I::p], b = B[i][I::q];
        B[i][I::p] = fmaf(c, a, ss_ * b);
        B[i][I::q] = fmaf(c, b, -ss_ * a);
    }
}

// entry (l, j) of [r x] with structurally-zero entries known at compile time;
// MASK bit 0/1/2 = r.x/r.y/r.z may be non-zero
template <int MASK>
__device__ __forceinline__ constexpr bool skew_nz(int l, int j) {
    return (l == 0 && j == 1 && (MASK & 4)) || (l == 0 && j == 2 && (MASK & 2)) ||
           (l == 1 && j == 0 && (MASK & 4)) || (l == 1 && j == 2 && (MASK & 1)) ||
           (l == 2 && j == 0 && (MASK & 2)) || (l == 2 && j == 1 && (MASK & 1));
}
template <int MASK>
__device__ __forceinline__ constexpr bool skew_row_nz(int i) {
    return skew_nz<MASK>(i, 0) || skew_nz<MASK>(i, 1) || skew_nz<MASK>(i, 2);
}
__device__ __forceinline__ float skew_at(float3 r, int l, int j) {
    return l == 0 ? (j == 1 ? -r.z : r.y) : (l == 1 ? (j == 0 ? r.z : -r.x) : (j == 0 ? -r.y : r.x));
}

// Congruence of a spatial inertia into the parent frame, X^T M X with
// X = rot(E) xlt(r) (joint about AX, then the joint origin r), plus, when ADD,
// the parent body's structured inertia I (expressed in the parent frame):
//   rotate every block by E^T, then
//   A'' = A' - P - P^T - Q,  B'' = B' + T,  C'' = C',
//   P = B' [r x],  T = [r x] C',  Q = T [r x],
// each A'' entry one FMA chain over its non-zero terms.  I's rotational part
// seeds the rotation chains of A (A' feeds only A''); its B and C parts are
// added once the translation has used B' and C'.
template <int AX, int MASK, bool ADD>
__device__ __forceinline__ void congruence(Sym6& M, float c, float s, float3 r, const BodyI& I) {
    rot_sym<AX, ADD>(M.A, c, s, f3(I.ax, I.ay, I.az));
    rot_gen<AX>(M.B, c, s);
    rot_sym<AX, false>(M.C, c, s, f3(0.f, 0.f, 0.f));
    float T[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float t = 0.f;
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (skew_nz<MASK>(i, l)) t = fmaf(skew_at(r, i, l), M.C[sidx(l, j)], t);
            T[i][j] = t;
        }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            float acc = M.A[sidx(i, j)];
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (skew_nz<MASK>(l, j)) acc = fmaf(-M.B[i][l], skew_at(r, l, j), acc);   // - P_ij
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (skew_nz<MASK>(l, i)) acc = fmaf(-M.B[j][l], skew_at(r, l, i), acc);   // - P_ji
#pragma unroll
            for (int l = 0; l < 3; l++)
                if (skew_row_nz<MASK>(i) && skew_nz<MASK>(l, j)) acc = fmaf(-T[i][l], skew_at(r, l, j), acc);  // - Q_ij
            M.A[sidx(i, j)] = acc;
        }
#pragma unroll
    for (int i = 0; i < 3; i++)
        if (skew_row_nz<MASK>(i))
#pragma unroll
            for (int j = 0; j < 3; j++) M.B[i][j] += T[i][j];
    if (ADD) {
        // I = [diag(a), m [c x]; m [c x]^T, m 1] with c = (0, 0, cz)
        M.B[0][1] -= I.mcz;
        M.B[1][0] += I.mcz;
        M.C[0] += I.m;
        M.C[3] += I.m;
        M.C[5] += I.m;
    }
}

// (ha, hl) += M [w; v] for a symmetric spatial matrix M and a spatial vector
// whose component AX (of both halves) is structurally zero
template <int AX>
__device__ __forceinline__ void sym6_mv_acc(const Sym6& M, float3 w, float3 v, float3& ha, float3& hl) {
    const float w_[3] = {w.x, w.y, w.z}, v_[3] = {v.x, v.y, v.z};
    float a[3] = {ha.x, ha.y, ha.z}, l[3] = {hl.x, hl.y, hl.z};
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (j == AX) continue;
            a[i] = fmaf(M.A[sidx(i, j)], w_[j], a[i]);
            a[i] = fmaf(M.B[i][j], v_[j], a[i]);
            l[i] = fmaf(M.B[j][i], w_[j], l[i]);
            l[i] = fmaf(M.C[sidx(i, j)], v_[j], l[i]);
        }
    ha = f3(a[0], a[1], a[2]);
    hl = f3(l[0], l[1], l[2]);
}

// I [w; v] for a body inertia with its centre of mass on the frame's z axis
__device__ __forceinline__ void bodyI_mv(const BodyI& I, float3 w, float3 v, float3& ha, float3& hl) {
    ha = f3(I.ax * w.x - I.mcz * v.y, I.ay * w.y + I.mcz * v.x, I.az * w.z);
    hl = f3(I.mcz * w.y + I.m * v.x, I.m * v.y - I.mcz * w.x, I.m * v.z);
}

// sin and cos of an angle |x| < 2^21: x = k pi + r with k the nearest integer to
// x / pi (rounded by the 1.5 * 2^23 shift, whose low mantissa bits then hold k),
// a two-term Cody-Waite reduction to |r| <= pi/2, Taylor polynomials to r^13 /
// r^12 (truncation below 7e-9), and the sign (-1)^k set by flipping sign bits.
__device__ __forceinline__ void sincos_r(float x, float& s, float& c) {
    const float t = fmaf(x, 0.318309886f, 12582912.f);
    const float k = t - 12582912.f;
    float r = fmaf(k, -3.14159274f, x);
    r = fmaf(k, 8.74227766e-08f, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 1.60590438e-10f, -2.50521084e-08f);
    ps = fmaf(r2, ps, 2.75573192e-06f);
    ps = fmaf(r2, ps, -1.98412698e-04f);
    ps = fmaf(r2, ps, 8.33333333e-03f);
    ps = fmaf(r2, ps, -1.66666667e-01f);
    const float sn = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, 2.08767570e-09f, -2.75573192e-07f);
    pc = fmaf(r2, pc, 2.48015873e-05f);
    pc = fmaf(r2, pc, -1.38888889e-03f);
    pc = fmaf(r2, pc, 4.16666667e-02f);
    pc = fmaf(r2, pc, -0.5f);
    const float cs = fmaf(r2, pc, 1.f);
    const unsigned sg = (unsigned)__float_as_int(t) << 31;
    s = __int_as_float(__float_as_int(sn) ^ (int)sg);
    c = __int_as_float(__float_as_int(cs) ^ (int)sg);
}

// rotation matrix (body -> world) of a unit quaternion (w, x, y, z):
// R = 1 + 2 w [v x] + 2 [v x]^2, each entry one short FMA chain
__device__ __forceinline__ void quat_R(const float q[4], float R[3][3]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float x2 = x + x, y2 = y + y, z2 = z + z;
    const float wx = w * x2, wy = w * y2, wz = w * z2;
    R[0][0] = fmaf(-y, y2, fmaf(-z, z2, 1.f));
    R[1][1] = fmaf(-x, x2, fmaf(-z, z2, 1.f));
    R[2][2] = fmaf(-x, x2, fmaf(-y, y2, 1.f));
    R[0][1] = fmaf(x, y2, -wz);
    R[1][0] = fmaf(x, y2, wz);
    R[0][2] = fmaf(x, z2, wy);
    R[2][0] = fmaf(x, z2, -wy);
    R[1][2] = fmaf(y, z2, -wx);
    R[2][1] = fmaf(y, z2, wx);
}
__device__ __forceinline__ float3 mulR(const float R[3][3], float3 v) {
    return f3(R[0][0] * v.x + R[0][1] * v.y + R[0][2] * v.z, R[1][0] * v.x + R[1][1] * v.y + R[1][2] * v.z,
              R[2][0] * v.x + R[2][1] * v.y + R[2][2] * v.z);
}
__device__ __forceinline__ float3 mulRT(const float R[3][3], float3 v) {
    return f3(R[0][0] * v.x + R[1][0] * v.y + R[2][0] * v.z, R[0][1] * v.x + R[1][1] * v.y + R[2][1] * v.z,
              R[0][2] * v.x + R[1][2] * v.y + R[2][2] * v.z);
}

}  // namespace mppi
