// rollout.cu -- K2: MPPI rollouts on sm_103a CUDA cores (FP32).
//
// arXiv 2409.10469, Alg. 1 inner loop: every sample's knot vector is turned into
// joint targets by the cubic spline (Sec. III-B), tracked by PD (Sec. IV-A) and
// simulated for T steps while L_walk (Sec. IV-B) and L_box (Sec. IV-D) accumulate.
// The simulator is the model spec's replacement for MuJoCo (Sec. III-A):
// floating-base articulated-body algorithm, penalty contacts with regularised
// Coulomb friction, semi-implicit Euler with n_sub sub-steps, implicit PD damping.
//
// Mapping: one rollout = 4 consecutive lanes, one lane per leg.  Each lane runs
// its leg's 3-body chain of every ABA pass in registers; the legs meet only at
// the trunk, whose articulated inertia (21 numbers) and bias force (6) are summed
// with two xor-shuffle rounds.  Every lane then holds bit-identical trunk sums and
// solves the 6x6 trunk system itself, so the replicated trunk state never
// diverges between lanes.  A warp holds 8 rollouts.
#include "common.cuh"
#include "kernels.h"

namespace mppi {

struct LegState {
    float q[3], qd[3];
};

struct Trunk {
    float p[3], quat[4];
    float3 w, v;  // body-frame angular and linear velocity
};

__device__ __forceinline__ float xsum4(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// ---------------------------------------------------------------- terrain

// ground height and slope under (x, y): plane, or bilinear heightfield with
// clamped edges (zero slope across a clamped edge)
template <int TERR>
__device__ __forceinline__ void ground(const DevModel& m, float x, float y, float& h, float& hx, float& hy) {
    if (TERR == 0) { h = 0.f; hx = 0.f; hy = 0.f; return; }
    float u = (x - m.hf_x0) * m.hf_inv_cell, v = (y - m.hf_y0) * m.hf_inv_cell;
    const float umax = (float)(m.hf_nx - 1), vmax = (float)(m.hf_ny - 1);
    bool inx = (u >= 0.f) && (u <= umax), iny = (v >= 0.f) && (v <= vmax);
    u = fminf(fmaxf(u, 0.f), umax);
    v = fminf(fmaxf(v, 0.f), vmax);
    int i = min((int)floorf(u), m.hf_nx - 2), j = min((int)floorf(v), m.hf_ny - 2);
    float fx = u - (float)i, fy = v - (float)j;
    const float* r0 = m.hf + j * m.hf_nx + i;
    float h00 = __ldg(r0), h10 = __ldg(r0 + 1), h01 = __ldg(r0 + m.hf_nx), h11 = __ldg(r0 + m.hf_nx + 1);
    h = (1.f - fx) * (1.f - fy) * h00 + fx * (1.f - fy) * h10 + (1.f - fx) * fy * h01 + fx * fy * h11;
    hx = inx ? ((1.f - fy) * (h10 - h00) + fy * (h11 - h01)) * m.hf_inv_cell : 0.f;
    hy = iny ? ((1.f - fx) * (h01 - h00) + fx * (h11 - h10)) * m.hf_inv_cell : 0.f;
}

// sphere vs axis-aligned box: outward normal and depth when overlapping
__device__ __forceinline__ bool sphere_aabb(float3 x, float r, float3 lo, float3 hi, float3& n, float& pen) {
    float3 cp = f3(fminf(fmaxf(x.x, lo.x), hi.x), fminf(fmaxf(x.y, lo.y), hi.y), fminf(fmaxf(x.z, lo.z), hi.z));
    float3 d = x - cp;
    float d2 = dot3(d, d);
    if (d2 > 0.f) {
        float dn = sqrtf(d2);
        if (dn >= r) return false;
        float inv = 1.f / dn;
        n = inv * d;
        pen = r - dn;
        return true;
    }
    // centre inside: leave through the nearest face (order x-, x+, y-, y+, z-, z+)
    float best = x.x - lo.x; int bf = 0;
    float t;
    t = hi.x - x.x; if (t < best) { best = t; bf = 1; }
    t = x.y - lo.y; if (t < best) { best = t; bf = 2; }
    t = hi.y - x.y; if (t < best) { best = t; bf = 3; }
    t = x.z - lo.z; if (t < best) { best = t; bf = 4; }
    t = hi.z - x.z; if (t < best) { best = t; bf = 5; }
    float sgn = (bf & 1) ? 1.f : -1.f;
    n = f3(bf / 2 == 0 ? sgn : 0.f, bf / 2 == 1 ? sgn : 0.f, bf / 2 == 2 ? sgn : 0.f);
    pen = r + best;
    return true;
}

// Force (in body coordinates) of one contact on a sphere fixed in a body.
// nb: normal in body coordinates, cb: sphere centre in the body frame, (w, v):
// body velocity; the force acts at the deepest point cb - r nb.
__device__ __forceinline__ void contact_wrench(const DevModel& m, float pen, float3 nb, float3 cb, float r,
                                               float3 w, float3 v, float3& torque, float3& force) {
    float3 pc = cb - r * nb;
    float3 vp = v + cross3(w, pc);
    float vn = dot3(vp, nb);
    float fn = fmaxf(m.kc * pen - m.cc * vn, 0.f);
    float3 vt = vp - vn * nb;
    float s = sqrtf(dot3(vt, vt) + m.eps2);
    float fr = m.mu * fn / s;
    float3 f = fn * nb - fr * vt;
    force = force + f;
    torque = torque + cross3(pc, f);
}

// all static-environment contacts of one sphere (world centre xw, radius r);
// RT(world) maps a world vector into the body's coordinates
template <int TERR, typename ToBody>
__device__ __forceinline__ void sphere_env(const DevModel& m, float3 xw, float r, float3 cb, float3 w, float3 v,
                                           ToBody toBody, float3& torque, float3& force) {
    float h, hx, hy;
    ground<TERR>(m, xw.x, xw.y, h, hx, hy);
    float inv = 1.f / sqrtf(hx * hx + hy * hy + 1.f);
    float3 n = f3(-hx * inv, -hy * inv, inv);
    float pen = r - (xw.z - h) * n.z;
    if (pen > 0.f) contact_wrench(m, pen, toBody(n), cb, r, w, v, torque, force);
    for (int b = 0; b < m.n_sbox; b++) {
        float3 nn; float pb;
        if (sphere_aabb(xw, r, ld3(m.sb_lo[b]), ld3(m.sb_hi[b]), nn, pb))
            contact_wrench(m, pb, toBody(nn), cb, r, w, v, torque, force);
    }
}

// ---------------------------------------------------------------- cost

__device__ __forceinline__ float trunk_state_cost(const DevCost& c, const Trunk& T) {
    float dz = T.p[2] - c.z_ref;
    float L = c.w_z * dz * dz;
    float sg = T.quat[0] < 0.f ? -2.f : 2.f;
    float ex = sg * T.quat[1], ey = sg * T.quat[2], ez = sg * T.quat[3];
    L += c.w_o * (ex * ex + ey * ey + ez * ez);
    float dv = T.v.x - c.v_ref;
    L += c.w_v * dv * dv;
    float dx = T.p[0] - c.goal_x, dy = T.p[1] - c.goal_y;
    L += c.w_p * (dx * dx + dy * dy);
    return L;
}

// ---------------------------------------------------------------- one sub-step

template <int TERR>
__device__ __forceinline__ void substep(const DevModel& m, int leg, Trunk& T, LegState& S, const float u[3],
                                        float h) {
    const float g = m.gz;
    float R0[3][3];
    quat_R(T.quat, R0);

    // ---- leg kinematics: joint transforms, body velocities, velocity products
    float c0, s0, c1, s1, c2, s2;
    sincosf(S.q[0], &s0, &c0);
    sincosf(S.q[1], &s1, &c1);
    sincosf(S.q[2], &s2, &c2);
    const float3 rh = ld3(m.r_hip[leg]), rt = ld3(m.r_thigh[leg]), rk = ld3(m.r_knee);
    // hip (axis x)
    float3 wh = Ex(c0, s0, T.w);
    float3 vh = Ex(c0, s0, T.v + cross3(T.w, rh));
    float3 ch_w = f3(0.f, wh.z * S.qd[0], -wh.y * S.qd[0]);   // w x (e_x qd)
    float3 ch_v = f3(0.f, vh.z * S.qd[0], -vh.y * S.qd[0]);
    wh.x += S.qd[0];
    // thigh (axis y)
    float3 wt = Ey(c1, s1, wh);
    float3 vt = Ey(c1, s1, vh + cross3(wh, rt));
    float3 ct_w = f3(-wt.z * S.qd[1], 0.f, wt.x * S.qd[1]);   // w x (e_y qd)
    float3 ct_v = f3(-vt.z * S.qd[1], 0.f, vt.x * S.qd[1]);
    wt.y += S.qd[1];
    // calf (axis y)
    float3 wc = Ey(c2, s2, wt);
    float3 vc = Ey(c2, s2, vt + cross3(wt, rk));
    float3 cc_w = f3(-wc.z * S.qd[2], 0.f, wc.x * S.qd[2]);
    float3 cc_v = f3(-vc.z * S.qd[2], 0.f, vc.x * S.qd[2]);
    wc.y += S.qd[2];

    // ---- contacts: the foot sphere on the calf
    float3 fc_n = f3(0.f, 0.f, 0.f), fc_f = f3(0.f, 0.f, 0.f);
    {
        const float3 foot = ld3(m.foot);
        float3 ptr = rh + ExT(c0, s0, rt + EyT(c1, s1, rk + EyT(c2, s2, foot)));   // trunk frame
        float3 xw = f3(T.p[0], T.p[1], T.p[2]) + mulR(R0, ptr);
        auto toCalf = [&](float3 nw) { return Ey(c2, s2, Ey(c1, s1, Ex(c0, s0, mulRT(R0, nw)))); };
        sphere_env<TERR>(m, xw, m.foot_r, foot, wc, vc, toCalf, fc_n, fc_f);
    }
    // ---- contacts: trunk spheres, one per lane, summed over the 4 lanes
    float3 f0_n = f3(0.f, 0.f, 0.f), f0_f = f3(0.f, 0.f, 0.f);
    if (leg < m.n_tsph) {
        float3 cb = f3(m.tsph_x[leg], 0.f, 0.f);
        float3 xw = f3(T.p[0], T.p[1], T.p[2]) + mulR(R0, cb);
        auto toTrunk = [&](float3 nw) { return mulRT(R0, nw); };
        sphere_env<TERR>(m, xw, m.tsph_r, cb, T.w, T.v, toTrunk, f0_n, f0_f);
    }

    // ---- PD with implicit damping: tau = kp (u - q - h qd) - kd qd, armature h (kd + h kp)
    const float arm = h * (m.kd + h * m.kp) + m.arm0;
    float tau[3];
#pragma unroll
    for (int i = 0; i < 3; i++) tau[i] = m.kp * (u[i] - S.q[i] - h * S.qd[i]) - m.kd * S.qd[i];

    // ---- pass 2 (tip to root), bias forces pA = v x* I v - f_ext
    float3 pa_n, pa_f;
    Sym6 IA;
    float U2[6], D2inv, u2, U1[6], D1inv, u1, U0[6], D0inv, u0;
    {   // calf
        IA = m.I_calf;
        float3 ha, hl;
        sym6_mv(IA, wc, vc, ha, hl);
        pa_n = cross3(wc, ha) + cross3(vc, hl) - fc_n;
        pa_f = cross3(wc, hl) - fc_f;
        U2[0] = IA.A[0][1]; U2[1] = IA.A[1][1]; U2[2] = IA.A[2][1];
        U2[3] = IA.B[1][0]; U2[4] = IA.B[1][1]; U2[5] = IA.B[1][2];
        D2inv = 1.f / (U2[1] + arm);
        u2 = tau[2] - pa_n.y;
    }
    // articulated quantities passed to the thigh
    auto project = [&](Sym6& M, float3& pn, float3& pf, const float U[6], float Dinv, float uu, float3 cw,
                       float3 cv) {
        // Ia = IA - U U^T / D ; pa = pA + Ia c + U u / D
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                M.A[i][j] -= U[i] * U[j] * Dinv;
                M.B[i][j] -= U[i] * U[3 + j] * Dinv;
                M.C[i][j] -= U[3 + i] * U[3 + j] * Dinv;
            }
        float3 ia, il;
        sym6_mv(M, cw, cv, ia, il);
        float k = uu * Dinv;
        pn = pn + ia + k * f3(U[0], U[1], U[2]);
        pf = pf + il + k * f3(U[3], U[4], U[5]);
    };
    project(IA, pa_n, pa_f, U2, D2inv, u2, cc_w, cc_v);
    // to the thigh frame: X^T pa = [E^T n + r x E^T f; E^T f]
    {
        float3 fn = EyT(c2, s2, pa_n), ff = EyT(c2, s2, pa_f);
        pa_n = fn + cross3(rk, ff);
        pa_f = ff;
        congruence<1>(IA, c2, s2, rk);
        sym6_add(IA, m.I_thigh);
        float3 ha, hl;
        sym6_mv(m.I_thigh, wt, vt, ha, hl);
        pa_n = pa_n + cross3(wt, ha) + cross3(vt, hl);
        pa_f = pa_f + cross3(wt, hl);
        U1[0] = IA.A[0][1]; U1[1] = IA.A[1][1]; U1[2] = IA.A[2][1];
        U1[3] = IA.B[1][0]; U1[4] = IA.B[1][1]; U1[5] = IA.B[1][2];
        D1inv = 1.f / (U1[1] + arm);
        u1 = tau[1] - pa_n.y;
    }
    project(IA, pa_n, pa_f, U1, D1inv, u1, ct_w, ct_v);
    {   // to the hip frame
        float3 fn = EyT(c1, s1, pa_n), ff = EyT(c1, s1, pa_f);
        pa_n = fn + cross3(rt, ff);
        pa_f = ff;
        congruence<1>(IA, c1, s1, rt);
        sym6_add(IA, m.I_hip);
        float3 ha, hl;
        sym6_mv(m.I_hip, wh, vh, ha, hl);
        pa_n = pa_n + cross3(wh, ha) + cross3(vh, hl);
        pa_f = pa_f + cross3(wh, hl);
        U0[0] = IA.A[0][0]; U0[1] = IA.A[1][0]; U0[2] = IA.A[2][0];
        U0[3] = IA.B[0][0]; U0[4] = IA.B[0][1]; U0[5] = IA.B[0][2];
        D0inv = 1.f / (U0[0] + arm);
        u0 = tau[0] - pa_n.x;
    }
    project(IA, pa_n, pa_f, U0, D0inv, u0, ch_w, ch_v);
    {   // to the trunk frame
        float3 fn = ExT(c0, s0, pa_n), ff = ExT(c0, s0, pa_f);
        pa_n = fn + cross3(rh, ff);
        pa_f = ff;
        congruence<0>(IA, c0, s0, rh);
    }

    // ---- trunk: sum the 4 legs' contributions, add the trunk's own terms
    float Mt[6][6], bt[6];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            Mt[i][j] = xsum4(IA.A[i][j]);
            Mt[3 + i][3 + j] = xsum4(IA.C[i][j]);
        }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Mt[i][3 + j] = xsum4(IA.B[i][j]);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Mt[i][i] += m.tr_Ic[i];
        Mt[3 + i][3 + i] += m.tr_m;
    }
    {
        // per-lane terms (leg bias, minus this lane's trunk-sphere wrench) summed
        // over the 4 lanes, then the trunk's own bias v x* I v once
        float3 Iw = f3(m.tr_Ic[0] * T.w.x, m.tr_Ic[1] * T.w.y, m.tr_Ic[2] * T.w.z);
        float3 bn = cross3(T.w, Iw), bf = m.tr_m * cross3(T.w, T.v);
        bt[0] = xsum4(pa_n.x - f0_n.x) + bn.x;
        bt[1] = xsum4(pa_n.y - f0_n.y) + bn.y;
        bt[2] = xsum4(pa_n.z - f0_n.z) + bn.z;
        bt[3] = xsum4(pa_f.x - f0_f.x) + bf.x;
        bt[4] = xsum4(pa_f.y - f0_f.y) + bf.y;
        bt[5] = xsum4(pa_f.z - f0_f.z) + bf.z;
    }
    // ---- solve Mt a' = -bt (Cholesky, 6x6 SPD)
    float Lc[6][6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        float d = Mt[j][j];
#pragma unroll
        for (int k = 0; k < j; k++) d -= Lc[j][k] * Lc[j][k];
        float ljj = sqrtf(d);
        float inv = 1.f / ljj;
        Lc[j][j] = ljj;
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            float sum = Mt[j][i];  // symmetric: (i, j) = (j, i), upper storage
#pragma unroll
            for (int k = 0; k < j; k++) sum -= Lc[i][k] * Lc[j][k];
            Lc[i][j] = sum * inv;
        }
    }
    float y[6], a0[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float sum = -bt[i];
#pragma unroll
        for (int k = 0; k < i; k++) sum -= Lc[i][k] * y[k];
        y[i] = sum / Lc[i][i];
    }
#pragma unroll
    for (int i = 5; i >= 0; i--) {
        float sum = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; k++) sum -= Lc[k][i] * a0[k];
        a0[i] = sum / Lc[i][i];
    }

    // ---- pass 3 (root to tip): a' = X a'_parent + c ; qdd = (u - U . a') / D
    float qdd[3];
    float3 aw = f3(a0[0], a0[1], a0[2]), av = f3(a0[3], a0[4], a0[5]);
    {
        float3 nw = Ex(c0, s0, aw), nv = Ex(c0, s0, av + cross3(aw, rh));
        nw = nw + ch_w; nv = nv + ch_v;
        qdd[0] = (u0 - (U0[0] * nw.x + U0[1] * nw.y + U0[2] * nw.z + U0[3] * nv.x + U0[4] * nv.y + U0[5] * nv.z)) * D0inv;
        nw.x += qdd[0];
        float3 tw = Ey(c1, s1, nw), tv = Ey(c1, s1, nv + cross3(nw, rt));
        tw = tw + ct_w; tv = tv + ct_v;
        qdd[1] = (u1 - (U1[0] * tw.x + U1[1] * tw.y + U1[2] * tw.z + U1[3] * tv.x + U1[4] * tv.y + U1[5] * tv.z)) * D1inv;
        tw.y += qdd[1];
        float3 kw = Ey(c2, s2, tw), kv = Ey(c2, s2, tv + cross3(tw, rk));
        kw = kw + cc_w; kv = kv + cc_v;
        qdd[2] = (u2 - (U2[0] * kw.x + U2[1] * kw.y + U2[2] * kw.z + U2[3] * kv.x + U2[4] * kv.y + U2[5] * kv.z)) * D2inv;
    }

    // ---- semi-implicit Euler
#pragma unroll
    for (int i = 0; i < 3; i++) {
        S.qd[i] += h * qdd[i];
        S.q[i] += h * S.qd[i];
    }
    float3 gb = f3(R0[2][0] * g, R0[2][1] * g, R0[2][2] * g);  // R0^T (0, 0, g)
    T.w = T.w + h * aw;
    T.v = T.v + h * (av + gb);
    float3 dp = mulR(R0, T.v);
    T.p[0] += h * dp.x; T.p[1] += h * dp.y; T.p[2] += h * dp.z;
    quat_integrate(T.quat, T.w, h);
}

// ---------------------------------------------------------------- kernel

template <int TERR, bool TRAJ>
__global__ void __launch_bounds__(256) k_rollout(RolloutArgs a) {
    const DevModel& m = a.model;
    const DevCost& c = a.cost;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt >> 2, leg = gt & 3;
    const bool valid = k < a.n;
    const int kk = valid ? k : a.n - 1;
    const int nx = m.nx;
    const float* x0 = a.x0 + (a.x0_per_sample ? (size_t)kk * nx : 0);

    Trunk T;
    T.p[0] = x0[0]; T.p[1] = x0[1]; T.p[2] = x0[2];
    T.quat[0] = x0[3]; T.quat[1] = x0[4]; T.quat[2] = x0[5]; T.quat[3] = x0[6];
    T.w = f3(x0[19], x0[20], x0[21]);
    T.v = f3(x0[22], x0[23], x0[24]);
    LegState S;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        S.q[i] = x0[7 + 3 * leg + i];
        S.qd[i] = x0[25 + 3 * leg + i];
    }
    float Uk[NKNOT][3];
    const float* Urow = a.U + (size_t)kk * D;
#pragma unroll
    for (int j = 0; j < NKNOT; j++)
#pragma unroll
        for (int i = 0; i < 3; i++) Uk[j][i] = Urow[j * NJ + 3 * leg + i];

    const float h = a.h;
    const float ph0 = (leg == 1 || leg == 2) ? 3.14159265358979f : 0.f;
    float L = 0.f;
    auto store = [&](int t) {
        if (!TRAJ || !valid) return;
        float* o = a.traj + ((size_t)k * (a.H + 1) + t) * nx;
        if (leg == 0) {
            o[0] = T.p[0]; o[1] = T.p[1]; o[2] = T.p[2];
            o[3] = T.quat[0]; o[4] = T.quat[1]; o[5] = T.quat[2]; o[6] = T.quat[3];
            o[19] = T.w.x; o[20] = T.w.y; o[21] = T.w.z;
            o[22] = T.v.x; o[23] = T.v.y; o[24] = T.v.z;
        }
#pragma unroll
        for (int i = 0; i < 3; i++) {
            o[7 + 3 * leg + i] = S.q[i];
            o[25 + 3 * leg + i] = S.qd[i];
        }
    };
    store(0);
    for (int t = 0; t < a.H; t++) {
        // cubic through 4 knots at tau_j = j / 3 (Lagrange basis)
        const float tau = (float)t * a.inv_Hm1;
        const float d0 = tau, d1 = tau - (1.f / 3.f), d2 = tau - (2.f / 3.f), d3 = tau - 1.f;
        const float B0 = d1 * d2 * d3 * -4.5f, B1 = d0 * d2 * d3 * 13.5f;
        const float B2 = d0 * d1 * d3 * -13.5f, B3 = d0 * d1 * d2 * 4.5f;
        float u[3];
#pragma unroll
        for (int i = 0; i < 3; i++) u[i] = B0 * Uk[0][i] + B1 * Uk[1][i] + B2 * Uk[2][i] + B3 * Uk[3][i];
        // stage cost: this leg's control term; the trunk terms on lane 0
        {
            float ds = 0.f, dk = 0.f;
            if (c.gait == 1) {
                float s = sinf(c.two_pi_over_period * (a.t0 + (float)t * a.dt) + ph0);
                ds = c.hip_amp * s;
                dk = -c.knee_amp * fmaxf(s, 0.f);
            }
            float e0 = u[0] - c.stand[0], e1 = u[1] - (c.stand[1] + ds), e2 = u[2] - (c.stand[2] + dk);
            L += c.w_u * (e0 * e0 + e1 * e1 + e2 * e2);
            if (leg == 0) L += trunk_state_cost(c, T);
        }
        for (int sidx = 0; sidx < a.n_sub; sidx++) substep<TERR>(m, leg, T, S, u, h);
        store(t + 1);
    }
    if (leg == 0) L += c.w_term * trunk_state_cost(c, T);
    L = xsum4(L);
    if (valid && leg == 0) a.L[k] = L;
}

template <int TERR, bool TRAJ>
static cudaError_t launch_t(const RolloutArgs& a, int block, cudaStream_t st) {
    long threads = 4L * a.n;
    int grid = (int)((threads + block - 1) / block);
    k_rollout<TERR, TRAJ><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rollout(const RolloutArgs& a, int block, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (a.model.terrain == 1)
        return a.traj ? launch_t<1, true>(a, block, st) : launch_t<1, false>(a, block, st);
    return a.traj ? launch_t<0, true>(a, block, st) : launch_t<0, false>(a, block, st);
}

}  // namespace mppi
