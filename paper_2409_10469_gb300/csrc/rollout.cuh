// rollout.cuh -- per-lane device code of the MPPI rollouts (arXiv 2409.10469,
// Alg. 1 inner loop; simulator per the model spec that replaces MuJoCo,
// Sec. III-A): terrain and contact geometry, L_walk / L_box stage costs, one
// semi-implicit sub-step of the floating-base ABA with PD and contacts, and
// the whole horizon of one rollout for one lane.  Shared by the single-instance
// kernel (rollout.cu) and the persistent multi-instance kernel (batch.cu), so
// both compute every rollout with the same arithmetic.
//
// Mapping: one rollout = 4 consecutive lanes, one lane per leg.  Each lane runs
// its leg's 3-body chain of every ABA pass in registers; the legs meet only at
// the trunk, whose articulated inertia (21 numbers) and bias force (6) are summed
// with two xor-shuffle rounds (two values per packed addition).  Every lane then
// holds bit-identical trunk sums and solves the 6x6 trunk system itself, so the
// replicated trunk state never diverges between lanes.
//
// Precision: the contact spheres' heights (and, against the free box, their
// positions in the box frame) are evaluated as FP32 pairs (precise.cuh) from
// joint angles and trunk / box positions that carry an FP32 compensation term
// (the rounding error of every sub-step's position update) through a dt step; at the end of each dt step the state is rounded to FP32,
// the granularity of every output (trajectories, costs).  The rest of the
// sub-step is plain FP32.
#pragma once
#include "common.cuh"
#include "precise.cuh"

namespace mppi {


struct LegState {
    float q[3], qd[3];
    float ql[3];  // compensation of q within a dt step (q + ql is the angle)
};

struct Trunk {
    float p[3], quat[4];
    float3 w, v;     // body-frame angular and linear velocity
    float pl[3];     // compensation of p within a dt step
    float quatl[4];  // compensation of quat within a dt step
    float qc;        // (|quat|^2 - 1) / 2 until the first sub-step normalises it
};

__device__ __forceinline__ float xsum4(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// xsum4 of two values at once: each round adds both by one packed FP32
// addition (two IEEE additions, each rounded as xsum4's), so a and b come out
// bit-identical to xsum4(a), xsum4(b) in half the add instructions
__device__ __forceinline__ void xsum4_pair(float& a, float& b) {
    float2 v = make_float2(a, b);
    v = __fadd2_rn(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1)));
    v = __fadd2_rn(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, 2), __shfl_xor_sync(0xffffffffu, v.y, 2)));
    a = v.x;
    b = v.y;
}

// ---------------------------------------------------------------- terrain

// ground height and slope under (x, y): plane, or bilinear heightfield with
// clamped edges (zero slope across a clamped edge)
__device__ __forceinline__ void ground(const DevModel& m, float x, float y, float& h, float& hx, float& hy) {
    if (m.terrain == 0) { h = 0.f; hx = 0.f; hy = 0.f; return; }
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

// terrain height under the point (x, y) given as pairs, as a pair (a cell
// corner's height and the bilinear correction, below 2e-2), and its slope.  The
// cell coordinate (x - x0) / cell is a pair too: the quotient's FP32 head and
// the remainder, which the FMA gives exactly, over the cell.  The same bilinear
// interpolation and edge clamping as ground().
__device__ __forceinline__ void ground_pair(const DevModel& m, F2 x, F2 y, F2& h, float& hx, float& hy) {
    if (m.terrain == 0) { h = F2{0.f, 0.f}; hx = 0.f; hy = 0.f; return; }
    const F2 dx = f2_addf(x, -m.hf_x0), dy = f2_addf(y, -m.hf_y0);
    const float qx = __fmul_rn(dx.h, m.hf_inv_cell), qy = __fmul_rn(dy.h, m.hf_inv_cell);
    const F2 u = two_sum(qx, __fmul_rn(__fadd_rn(__fmaf_rn(-qx, m.hf_cell, dx.h), dx.l), m.hf_inv_cell));
    const F2 v = two_sum(qy, __fmul_rn(__fadd_rn(__fmaf_rn(-qy, m.hf_cell, dy.h), dy.l), m.hf_inv_cell));
    const float umax = (float)(m.hf_nx - 1), vmax = (float)(m.hf_ny - 1);
    const bool inx = (u.h >= 0.f) && (u.h <= umax), iny = (v.h >= 0.f) && (v.h <= vmax);
    const float uc = fminf(fmaxf(u.h, 0.f), umax), vc = fminf(fmaxf(v.h, 0.f), vmax);
    const int i = min((int)floorf(uc), m.hf_nx - 2), j = min((int)floorf(vc), m.hf_ny - 2);
    const float fx = __fadd_rn(uc - (float)i, inx ? u.l : 0.f), fy = __fadd_rn(vc - (float)j, iny ? v.l : 0.f);
    const float* r0 = m.hf + j * m.hf_nx + i;
    const float h00 = __ldg(r0), h10 = __ldg(r0 + 1), h01 = __ldg(r0 + m.hf_nx), h11 = __ldg(r0 + m.hf_nx + 1);
    // (1-fx)(1-fy) h00 + fx (1-fy) h10 + (1-fx) fy h01 + fx fy h11 = h00 + fx ax + fy (ay + fx axy)
    const float ax = h10 - h00, ay = h01 - h00, axy = (h11 - h10) - ay;
    h = F2{h00, fmaf(fx, ax, fy * fmaf(fx, axy, ay))};
    hx = inx ? ((1.f - fy) * ax + fy * (h11 - h01)) * m.hf_inv_cell : 0.f;
    hy = iny ? ((1.f - fx) * ay + fx * (h11 - h10)) * m.hf_inv_cell : 0.f;
}

// sphere vs axis-aligned box: outward normal and depth when overlapping; xl is
// the low part of the centre (pairs x + xl), which enters the distance to the
// faces it lies beyond
__device__ __forceinline__ bool sphere_aabb(float3 x, float r, float3 lo, float3 hi, float3& n, float& pen,
                                            float3 xl = make_float3(0.f, 0.f, 0.f)) {
    float3 cp = f3(fminf(fmaxf(x.x, lo.x), hi.x), fminf(fmaxf(x.y, lo.y), hi.y), fminf(fmaxf(x.z, lo.z), hi.z));
    float3 d = x - cp;
    d.x += (x.x < lo.x || x.x > hi.x) ? xl.x : 0.f;
    d.y += (x.y < lo.y || x.y > hi.y) ? xl.y : 0.f;
    d.z += (x.z < lo.z || x.z > hi.z) ? xl.z : 0.f;
    float d2 = dot3(d, d);
    if (d2 > 0.f) {
        const float inv = rsqrtf(d2);   // approximate, branch-free (no IEEE slow path)
        const float dn = d2 * inv;
        if (dn >= r) return false;
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

// Force (in body coordinates) of one contact on a sphere fixed in a body, added
// to (torque, force) with sign SG (+1 a wrench on the body, -1 its negation as
// it enters a bias force).  nb: normal in body coordinates, cb: sphere centre
// in the body frame, (w, v): body velocity; the force acts at the deepest point
// cb - r nb.  An inactive contact adds exactly zero.
template <int SG>
__device__ __forceinline__ void contact_wrench(const DevModel& m, float pen, float3 nb, float3 cb, float r,
                                               float3 w, float3 v, float3& torque, float3& force,
                                               bool active = true) {
    const float3 pc = f3(fmaf(-r, nb.x, cb.x), fmaf(-r, nb.y, cb.y), fmaf(-r, nb.z, cb.z));
    const float3 vp = cross_acc(w, pc, v);
    const float vn = dot3(vp, nb);
    const float fn = active ? fmaxf(fmaf(m.kc, pen, -m.cc * vn), 0.f) : 0.f;
    const float3 vt = f3(fmaf(-vn, nb.x, vp.x), fmaf(-vn, nb.y, vp.y), fmaf(-vn, nb.z, vp.z));
    const float fr = m.mu * fn * rsqrt_approx(fmaf(vt.x, vt.x, fmaf(vt.y, vt.y, fmaf(vt.z, vt.z, m.eps2))));
    const float sn = SG > 0 ? fn : -fn, st = SG > 0 ? -fr : fr;
    const float3 f = f3(fmaf(sn, nb.x, st * vt.x), fmaf(sn, nb.y, st * vt.y), fmaf(sn, nb.z, st * vt.z));
    force = force + f;
    torque = cross_acc(pc, f, torque);
}

// world -> body coordinate maps of the two kinds of contact-sphere bodies
struct TrunkFrame {
    float r00, r01, r02, r10, r11, r12, r20, r21, r22;  // R0 (body -> world)
    __device__ __forceinline__ float3 operator()(float3 n) const {
        return f3(r00 * n.x + r10 * n.y + r20 * n.z, r01 * n.x + r11 * n.y + r21 * n.z,
                  r02 * n.x + r12 * n.y + r22 * n.z);
    }
    __device__ __forceinline__ float3 world(float3 v) const {
        return f3(r00 * v.x + r01 * v.y + r02 * v.z, r10 * v.x + r11 * v.y + r12 * v.z,
                  r20 * v.x + r21 * v.y + r22 * v.z);
    }
    __device__ __forceinline__ float3 ez() const { return f3(r20, r21, r22); }  // world e_z in body coordinates
};
struct CalfFrame {
    float r00, r01, r02, r10, r11, r12, r20, r21, r22;
    float c0, s0, c1, s1, c2, s2;
    __device__ __forceinline__ float3 operator()(float3 n) const {
        float3 t = f3(r00 * n.x + r10 * n.y + r20 * n.z, r01 * n.x + r11 * n.y + r21 * n.z,
                      r02 * n.x + r12 * n.y + r22 * n.z);
        return Ey(c2, s2, Ey(c1, s1, Ex(c0, s0, t)));
    }
    __device__ __forceinline__ float3 world(float3 v) const {
        float3 t = ExT(c0, s0, EyT(c1, s1, EyT(c2, s2, v)));
        return f3(r00 * t.x + r01 * t.y + r02 * t.z, r10 * t.x + r11 * t.y + r12 * t.z,
                  r20 * t.x + r21 * t.y + r22 * t.z);
    }
    __device__ __forceinline__ float3 ez() const { return Ey(c2, s2, Ey(c1, s1, Ex(c0, s0, f3(r20, r21, r22)))); }
};

// the free box of the push task: pose, rotation (box -> world) and body velocity
struct BoxState {
    float p[3], quat[4];
    float3 w, v;
    float pl[3];     // compensation of p within a dt step
    float quatl[4];  // compensation of quat within a dt step
    float qc;        // (|quat|^2 - 1) / 2 until the first sub-step normalises it
};
struct BoxKin {
    float3 p;
    float R[3][3];
    float3 w, v;
    F2 rz[3];   // row 2 of R as pairs (the corner spheres' heights)
};

// robot sphere (world centre xw, radius r, centre cb in its body) against the
// free box (oriented box in its own frame): equal and opposite forces at the
// sphere's deepest point, from the relative velocity of the two body points.
// An FP32 test first drops the spheres that cannot reach the box (its error,
// ~1e-6 m, is far inside the 1e-4 m margin); a sphere within reach enters the
// box frame as pairs, R^T (x - p) with the centre (pos(): its world position as
// pairs), the box's position and the rows of R as pairs -- a difference of
// ~0.5 m terms, as for the ground: FP32 would leave ~3e-8 m on the depth.  The
// robot's share goes to (torque, force) with sign SG, the box's to (bt, bf).
template <int SG, typename Frame, typename PairPos>
__device__ __forceinline__ void sphere_vs_box(const DevModel& m, const BoxKin& B, const BoxState& Bx, float3 xw,
                                              float r, float3 cb, float3 w, float3 v, const Frame& F,
                                              float3& torque, float3& force, float3& bt, float3& bf,
                                              const PairPos& pos, bool on = true) {
    const float3 hb = f3(m.box_half[0], m.box_half[1], m.box_half[2]);
    const float3 x32 = mulRT(B.R, xw - B.p);
    const float reach = r + 1e-4f;
    if (!on || fabsf(x32.x) > hb.x + reach || fabsf(x32.y) > hb.y + reach || fabsf(x32.z) > hb.z + reach) return;
    F2 xp, yp, zp;
    pos(xp, yp, zp);
    F2 brx[3], bry[3];
    quat_rows01(Bx.quat, Bx.quatl, brx, bry);
    const F2 dx = f2_sub(xp, F2{Bx.p[0], Bx.pl[0]}), dy = f2_sub(yp, F2{Bx.p[1], Bx.pl[1]});
    const F2 dz = f2_sub(zp, F2{Bx.p[2], Bx.pl[2]});
    F2 xq[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        xq[k] = f2_norm(f2_add(f2_add(f2_mul(brx[k], dx), f2_mul(bry[k], dy)), f2_mul(B.rz[k], dz)));
    const float3 xl = f3(xq[0].h, xq[1].h, xq[2].h);
    float3 nl;
    float pen;
    if (!sphere_aabb(xl, r, -hb, hb, nl, pen, f3(xq[0].l, xq[1].l, xq[2].l))) return;
    const float3 nw = mulR(B.R, nl);
    const float3 nb = F(nw);
    const float3 pc_b = cb - r * nb;                      // contact point, robot body frame
    const float3 vr_w = F.world(v + cross3(w, pc_b));
    const float3 pc_l = xl - r * nl;                      // contact point, box frame
    const float3 vb_w = mulR(B.R, B.v + cross3(B.w, pc_l));
    const float3 vrel = vr_w - vb_w;
    const float vn = dot3(vrel, nw);
    const float fn = fmaxf(m.kc * pen - m.cc * vn, 0.f);
    const float3 vt = vrel - vn * nw;
    const float fr = m.mu * fn * rsqrt_approx(dot3(vt, vt) + m.eps2);
    const float3 fw = fn * nw - fr * vt;
    const float3 fbody = SG > 0 ? F(fw) : -F(fw);
    force = force + fbody;
    torque = torque + cross3(pc_b, fbody);
    const float3 fl = -mulRT(B.R, fw);
    bf = bf + fl;
    bt = bt + cross3(pc_l, fl);
}

// All static-environment contacts of one sphere (world centre xw, radius r),
// added with sign SG; toBody maps a world vector into the body's coordinates.
// (xp, yp, zp) is the centre as pairs (xw its FP32 value), from which the depths
// are taken: flat ground needs only the height; over a heightfield and against
// static boxes the horizontal position places the sphere too.  TERR 0: flat
// ground and no static boxes (normal e_z, depth r - z); TERR 1: the model's
// plane or heightfield and its static boxes.  A sphere that is not `on` adds
// exactly zero.
template <int TERR, int SG, typename ToBody>
__device__ __forceinline__ void sphere_env(const DevModel& m, float3 xw, F2 xp, F2 yp, F2 zw, float r, float3 cb,
                                           float3 w, float3 v, const ToBody& toBody, float3& torque,
                                           float3& force, bool on = true) {
    if (TERR == 0) {
        const float pen = (r - zw.h) - zw.l;
        contact_wrench<SG>(m, fmaxf(pen, 0.f), toBody.ez(), cb, r, w, v, torque, force, on && pen > 0.f);
        return;
    }
    F2 hp;
    float hx, hy;
    ground_pair(m, xp, yp, hp, hx, hy);
    float inv = rsqrt_approx(hx * hx + hy * hy + 1.f);
    float3 n = f3(-hx * inv, -hy * inv, inv);
    const float pen = r - ((zw.h - hp.h) + (zw.l - hp.l)) * n.z;
    // the centre renormalised (FP32 values and low parts of under an ulp) for the
    // box tests, which compare it against the faces in FP32
    const F2 xn = f2_norm(xp), yn = f2_norm(yp), zn = f2_norm(zw);
    xw = f3(xn.h, yn.h, zn.h);
    // computed unconditionally and zeroed out of contact (no branch)
    contact_wrench<SG>(m, fmaxf(pen, 0.f), toBody(n), cb, r, w, v, torque, force, on && pen > 0.f);
    for (int b = 0; b < m.n_sbox; b++) {
        float3 nn; float pb;
        const float* bx = m.sbox + 6 * b;
        const float3 lo = f3(bx[0], bx[1], bx[2]);
        const float3 hi = f3(bx[3], bx[4], bx[5]);
        if (on && sphere_aabb(xw, r, lo, hi, nn, pb, f3(xn.l, yn.l, zn.l)))
            contact_wrench<SG>(m, pb, toBody(nn), cb, r, w, v, torque, force);
    }
}

// ---------------------------------------------------------------- cost

// height of the ground under (x, y): the plane or heightfield, or the top of a
// static box whose footprint contains (x, y), whichever is higher
__device__ __forceinline__ float ground_under(const DevModel& m, float x, float y) {
    float h, hx, hy;
    ground(m, x, y, h, hx, hy);
    for (int b = 0; b < m.n_sbox; b++) {
        const float* bx = m.sbox + 6 * b;
        if (x >= bx[0] && x <= bx[3] && y >= bx[1] && y <= bx[4]) h = fmaxf(h, bx[5]);
    }
    return h;
}

template <int TERR>
__device__ __forceinline__ float trunk_state_cost(const DevModel& m, const DevCost& c, const Trunk& T) {
    float dz = T.p[2] - c.z_ref;
    if (TERR != 0 && c.z_rel) dz -= ground_under(m, T.p[0], T.p[1]);   // flat ground without boxes: 0
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

// L_box (Sec. IV-D): Q_box times the l1 distance of the box to its goal (xy)
__device__ __forceinline__ float box_cost(const DevCost& c, const BoxState& B) {
    return c.w_box * (fabsf(c.box_gx - B.p[0]) + fabsf(c.box_gy - B.p[1]));
}

// ---------------------------------------------------------------- one sub-step

// velocity-product term c = v x (e_AX qd) of a joint about AX, from the body's
// velocity before its own joint rate is added (the joint's own part drops out)
template <int AX> __device__ __forceinline__ float3 vprod(float3 a, float qd) {
    return AX == 0 ? f3(0.f, a.z * qd, -a.y * qd) : f3(-a.z * qd, 0.f, a.x * qd);
}
// E v + c for such a term c of the same joint (its component on the joint axis
// is structurally zero), as two FMA chains per rotated component
__device__ __forceinline__ float3 Ex_vp(float c, float s, float3 v, float3 cv) {
    return f3(v.x, fmaf(c, v.y, fmaf(s, v.z, cv.y)), fmaf(c, v.z, fmaf(-s, v.y, cv.z)));
}
__device__ __forceinline__ float3 Ey_vp(float c, float s, float3 v, float3 cv) {
    return f3(fmaf(c, v.x, fmaf(-s, v.z, cv.x)), v.y, fmaf(s, v.x, fmaf(c, v.z, cv.z)));
}

// Ia = IA - U U^T / D  and  pa = pA + Ia c + U u / D for a joint about AX
// (U = IA e_AX); c has zero entries on the joint axis (structure of vprod).
template <int AX>
__device__ __forceinline__ void project(Sym6& M, float3& pn, float3& pf, float Dinv, float uu, float3 cw, float3 cv) {
    float Ua[3], Ul[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Ua[i] = M.A[sidx(i, AX)];
        Ul[i] = M.B[AX][i];
    }
    float Uas[3], Uls[3];
#pragma unroll
    for (int i = 0; i < 3; i++) { Uas[i] = Ua[i] * Dinv; Uls[i] = Ul[i] * Dinv; }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            M.A[sidx(i, j)] = fmaf(-Uas[i], Ua[j], M.A[sidx(i, j)]);
            M.C[sidx(i, j)] = fmaf(-Uls[i], Ul[j], M.C[sidx(i, j)]);
        }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M.B[i][j] = fmaf(-Uas[i], Ul[j], M.B[i][j]);
    sym6_mv_acc<AX>(M, cw, cv, pn, pf);
    const float k = uu * Dinv;
    pn = f3(fmaf(k, Ua[0], pn.x), fmaf(k, Ua[1], pn.y), fmaf(k, Ua[2], pn.z));
    pf = f3(fmaf(k, Ul[0], pf.x), fmaf(k, Ul[1], pf.y), fmaf(k, Ul[2], pf.z));
}

// bias force v x* I v of a body with a structured inertia, added to (bn, bf)
__device__ __forceinline__ void body_bias_acc(const BodyI& I, float3 w, float3 v, float3& bn, float3& bf) {
    float3 ha, hl;
    bodyI_mv(I, w, v, ha, hl);
    bn = cross_acc(v, hl, cross_acc(w, ha, bn));
    bf = cross_acc(w, hl, bf);
}

// Spatial force p in a child frame (joint about AX at angle (c, s), joint
// origin r in the parent) to the parent: X^T p = [E^T n + r x E^T f; E^T f].
// The origins of the knee (0, 0, rz) and the flexion joint (0, ry, 0) lie on a
// coordinate axis; the abduction joint's origin is general.
__device__ __forceinline__ void force_up_knee(float c, float s, float rz, float3& n, float3& f) {
    const float3 fn = EyT(c, s, n), ff = EyT(c, s, f);
    n = cross_z_acc(ff, -rz, fn);     // fn + (0, 0, rz) x ff
    f = ff;
}
__device__ __forceinline__ void force_up_flex(float c, float s, float ry, float3& n, float3& f) {
    const float3 fn = EyT(c, s, n), ff = EyT(c, s, f);
    n = cross_y_acc(ff, -ry, fn);     // fn + (0, ry, 0) x ff
    f = ff;
}
__device__ __forceinline__ void force_up_abd(float c, float s, float3 r, float3& n, float3& f) {
    const float3 fn = ExT(c, s, n), ff = ExT(c, s, f);
    n = cross_acc(r, ff, fn);
    f = ff;
}

// The leg-dependent constants of a lane, computed once per rollout (outside the
// time loops): legs FR, FL, RR, RL -- front (+x) for legs 0, 1, left (+y) for odd
// legs -- and the trunk sphere this lane carries (lanes past the last sphere
// carry none).
struct LegGeom {
    float3 rh;   // abduction joint in the trunk frame
    float ty;    // flexion joint (0, ty, 0) in the hip frame
    float tx;    // this lane's trunk sphere on the trunk x axis
    bool tsph;   // whether this lane carries a trunk sphere
};

__device__ __forceinline__ LegGeom leg_geom(const DevModel& m, int leg) {
    const float fx = leg < 2 ? 1.f : -1.f, sy = (leg & 1) ? 1.f : -1.f;
    LegGeom g;
    g.rh = f3(fx * m.hip_x, sy * m.hip_y, m.hip_z);
    g.ty = sy * m.thigh_y;
    g.tsph = leg < m.n_tsph;
    g.tx = leg == 0 ? m.tsph_x[0] : (leg == 1 ? m.tsph_x[1] : (leg == 2 ? m.tsph_x[2] : m.tsph_x[3]));
    return g;
}

// p += h dp with the height's rounding error (and, over terrain or with the
// free box, the horizontal ones: the heightfield and the static boxes are looked
// up at x, y, and robot spheres meet the box sideways) kept in pl
template <bool XY>
__device__ __forceinline__ void advance_pos(float p[3], float pl[3], float3 dp, float h) {
    const float d[3] = {dp.x, dp.y, dp.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (!XY && k < 2) {
            p[k] = fmaf(h, d[k], p[k]);
            continue;
        }
        const F2 t = fast_two_sum(p[k], h * d[k]);
        p[k] = t.h;
        pl[k] += t.l;
    }
}

// the state rounded to FP32 at the end of a dt step: every compensation term
// folded into its value, and the rounded quaternions' norm errors taken for the
// next sub-step's normalisation
template <bool BOX>
__device__ __forceinline__ void round_state(Trunk& T, LegState& S, BoxState& Bx) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T.p[k] += T.pl[k];
        T.pl[k] = 0.f;
        S.q[k] += S.ql[k];
        S.ql[k] = 0.f;
        if (BOX) {
            Bx.p[k] += Bx.pl[k];
            Bx.pl[k] = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        T.quat[k] += T.quatl[k];
        T.quatl[k] = 0.f;
        if (BOX) {
            Bx.quat[k] += Bx.quatl[k];
            Bx.quatl[k] = 0.f;
        }
    }
    T.qc = quat_half_norm_err(T.quat);
    if (BOX) Bx.qc = quat_half_norm_err(Bx.quat);
}

template <int TERR, bool BOX>
__device__ __forceinline__ void substep(const DevModel& m, int leg, const LegGeom& G, Trunk& T, LegState& S,
                                        const float kpu[3], float h, float kdh, float hg, float arm, BoxState& Bx) {
    const float g = m.gz;
    float R0[3][3];
    quat_R(T.quat, R0);
    BoxKin BK;
    float3 bx_t = f3(0.f, 0.f, 0.f), bx_f = f3(0.f, 0.f, 0.f);  // this lane's share of the box wrench
    if (BOX) {
        BK.p = f3(Bx.p[0], Bx.p[1], Bx.p[2]);
        quat_R(Bx.quat, BK.R);
        BK.w = Bx.w;
        BK.v = Bx.v;
        quat_row2(Bx.quat, Bx.quatl, BK.rz[0], BK.rz[1], BK.rz[2]);
    }

    // ---- leg kinematics: joint transforms, body velocities, velocity products.
    // Sines and cosines of the compensated angles as pairs (the FP32 values
    // serve the dynamics, the pairs the sphere heights), with q1 + q2 for the
    // foot's height: the knee and foot offsets lie on the thigh's and calf's z
    // axes, so in the hip frame the foot sits at
    // (kz sin q1 + fz sin q12, ty, kz cos q1 + fz cos q12)
    F2 S0p, C0p, S1p, C1p, S2p, C2p, S12p, C12p;
    sincos_pair(S.q[0], S.ql[0], S0p, C0p);
    sincos_pair(S.q[1], S.ql[1], S1p, C1p);
    sincos_pair(S.q[2], S.ql[2], S2p, C2p);
    {
        const F2 q12 = f2_add(F2{S.q[1], S.ql[1]}, F2{S.q[2], S.ql[2]});
        sincos_pair(q12.h, q12.l, S12p, C12p);
    }
    const float c0 = f2_val(C0p), s0 = f2_val(S0p), c1 = f2_val(C1p), s1 = f2_val(S1p);
    const float c2 = f2_val(C2p), s2 = f2_val(S2p);
    // the world's vertical in trunk coordinates, as pairs (sphere heights)
    F2 rz0, rz1, rz2;
    quat_row2(T.quat, T.quatl, rz0, rz1, rz2);
    const F2 pz_t = {T.p[2], T.pl[2]};
    // over terrain the spheres' horizontal positions as pairs too (rows 0 and 1;
    // against the free box they are formed only for spheres within its reach)
    F2 rx[3], ry[3];
    if (TERR != 0) quat_rows01(T.quat, T.quatl, rx, ry);
    const F2 px_t = {T.p[0], T.pl[0]}, py_t = {T.p[1], T.pl[1]};
    const float3 rh = G.rh;                                        // abduction joint in the trunk
    const float ty = G.ty;                                         // flexion joint (0, ty, 0) in the hip
    const float kz = m.r_knee[2], fz = m.foot[2];                  // knee (0, 0, kz), foot (0, 0, fz)
    float3 wh = Ex(c0, s0, T.w);
    float3 vh = Ex(c0, s0, cross_acc(T.w, rh, T.v));
    const float3 ch_w = vprod<0>(wh, S.qd[0]), ch_v = vprod<0>(vh, S.qd[0]);
    wh.x += S.qd[0];
    float3 wt = Ey(c1, s1, wh);
    float3 vt = Ey(c1, s1, cross_y_acc(wh, ty, vh));
    const float3 ct_w = vprod<1>(wt, S.qd[1]), ct_v = vprod<1>(vt, S.qd[1]);
    wt.y += S.qd[1];
    float3 wc = Ey(c2, s2, wt);
    float3 vc = Ey(c2, s2, cross_z_acc(wt, kz, vt));
    const float3 cc_w = vprod<1>(wc, S.qd[2]), cc_v = vprod<1>(vc, S.qd[2]);
    wc.y += S.qd[2];

    // ---- PD with implicit damping: tau = kp (u - q - h qd) - kd qd, armature h (kd + h kp);
    // kpu = kp u per dt step, kdh = kp h + kd per horizon
    float tau[3];
#pragma unroll
    for (int i = 0; i < 3; i++) tau[i] = fmaf(-kdh, S.qd[i], fmaf(-m.kp, S.q[i], fmaf(-m.kp, S.ql[i], kpu[i])));

    // ---- pass 2 (tip to root), calf: its bias minus the foot's contact wrench
    float3 pa_n = f3(0.f, 0.f, 0.f), pa_f = f3(0.f, 0.f, 0.f);
    body_bias_acc(m.I_calf, wc, vc, pa_n, pa_f);
    {
        const float3 foot = f3(0.f, 0.f, fz);
        // foot centre in the trunk frame: rh + E0^T ((0, ty, 0) + E1^T ((0, 0, kz) + E2^T foot)),
        // as pairs, and its world height p_z + (row 2 of R0) . ptr
        const F2 bx = f2_add(f2_mulf(S12p, fz), f2_mulf(S1p, kz));
        const F2 bz = f2_add(f2_mulf(C12p, fz), f2_mulf(C1p, kz));
        const F2 px = f2_addf(bx, rh.x);
        const F2 py = f2_sub(f2_addf(f2_mulf(C0p, ty), rh.y), f2_mul(S0p, bz));
        const F2 pz = f2_add(f2_addf(f2_mulf(S0p, ty), rh.z), f2_mul(C0p, bz));
        const F2 zw = f2_add(f2_add(pz_t, f2_mul(rz0, px)), f2_add(f2_mul(rz1, py), f2_mul(rz2, pz)));
        const float3 ptr = f3(f2_val(px), f2_val(py), f2_val(pz));
        const float3 xw = f3(T.p[0], T.p[1], T.p[2]) + mulR(R0, ptr);
        F2 xpw = {xw.x, 0.f}, ypw = {xw.y, 0.f};
        if (TERR != 0) {
            xpw = f2_add(f2_add(px_t, f2_mul(rx[0], px)), f2_add(f2_mul(rx[1], py), f2_mul(rx[2], pz)));
            ypw = f2_add(f2_add(py_t, f2_mul(ry[0], px)), f2_add(f2_mul(ry[1], py), f2_mul(ry[2], pz)));
        }
        const CalfFrame toCalf = {R0[0][0], R0[0][1], R0[0][2], R0[1][0], R0[1][1], R0[1][2],
                                  R0[2][0], R0[2][1], R0[2][2], c0, s0, c1, s1, c2, s2};
        sphere_env<TERR, -1>(m, xw, xpw, ypw, zw, m.foot_r, foot, wc, vc, toCalf, pa_n, pa_f);
        if (BOX) {
            const auto foot_pos = [&](F2& X, F2& Y, F2& Z) {
                if (TERR != 0) {
                    X = xpw;
                    Y = ypw;
                } else {
                    F2 qx[3], qy[3];
                    quat_rows01(T.quat, T.quatl, qx, qy);
                    X = f2_add(f2_add(px_t, f2_mul(qx[0], px)), f2_add(f2_mul(qx[1], py), f2_mul(qx[2], pz)));
                    Y = f2_add(f2_add(py_t, f2_mul(qy[0], px)), f2_add(f2_mul(qy[1], py), f2_mul(qy[2], pz)));
                }
                Z = zw;
            };
            sphere_vs_box<-1>(m, BK, Bx, xw, m.foot_r, foot, wc, vc, toCalf, pa_n, pa_f, bx_t, bx_f, foot_pos);
        }
    }
    // the calf's articulated inertia after projection is a model constant
    const float D2inv = m.calf_D_inv;
    const float u2 = tau[2] - pa_n.y;
    // U2 = I_calf e_y = (0, ay, 0 | mcz, 0, 0)
    const float U2a = m.I_calf.ay, U2l = m.I_calf.mcz;
    {
        sym6_mv_acc<1>(m.Ia_calf, cc_w, cc_v, pa_n, pa_f);
        const float k = u2 * D2inv;
        pa_n.y = fmaf(k, U2a, pa_n.y);
        pa_f.x = fmaf(k, U2l, pa_f.x);
    }
    // to the thigh frame
    Sym6 IA = m.Ia_calf;
    float U1a[3], U1l[3], D1inv, u1;
    {
        force_up_knee(c2, s2, kz, pa_n, pa_f);
        congruence<1, 4, true>(IA, c2, s2, f3(0.f, 0.f, kz), m.I_thigh);
        body_bias_acc(m.I_thigh, wt, vt, pa_n, pa_f);
#pragma unroll
        for (int i = 0; i < 3; i++) { U1a[i] = IA.A[sidx(i, 1)]; U1l[i] = IA.B[1][i]; }
        D1inv = rcp_approx(U1a[1] + arm);
        u1 = tau[1] - pa_n.y;
    }
    project<1>(IA, pa_n, pa_f, D1inv, u1, ct_w, ct_v);
    float U0a[3], U0l[3], D0inv, u0;
    {   // to the hip frame
        force_up_flex(c1, s1, ty, pa_n, pa_f);
        congruence<1, 2, true>(IA, c1, s1, f3(0.f, ty, 0.f), m.I_hip);
        body_bias_acc(m.I_hip, wh, vh, pa_n, pa_f);
#pragma unroll
        for (int i = 0; i < 3; i++) { U0a[i] = IA.A[sidx(i, 0)]; U0l[i] = IA.B[0][i]; }
        D0inv = rcp_approx(U0a[0] + arm);
        u0 = tau[0] - pa_n.x;
    }
    project<0>(IA, pa_n, pa_f, D0inv, u0, ch_w, ch_v);
    // to the trunk frame
    force_up_abd(c0, s0, rh, pa_n, pa_f);
    congruence<0, 7, false>(IA, c0, s0, rh, m.I_hip);

    // ---- contacts of the trunk spheres, one per lane (lanes past the last
    // sphere compute a zero wrench), minus into this lane's trunk bias
    {
        const bool on = G.tsph;
        const float tx = G.tx;
        const float3 cb = f3(tx, 0.f, 0.f);
        const float3 xw = f3(fmaf(R0[0][0], tx, T.p[0]), fmaf(R0[1][0], tx, T.p[1]), fmaf(R0[2][0], tx, T.p[2]));
        const F2 zw = f2_add(pz_t, f2_mulf(rz0, tx));
        const F2 xpw = TERR != 0 ? f2_add(px_t, f2_mulf(rx[0], tx)) : F2{xw.x, 0.f};
        const F2 ypw = TERR != 0 ? f2_add(py_t, f2_mulf(ry[0], tx)) : F2{xw.y, 0.f};
        const TrunkFrame toTrunk = {R0[0][0], R0[0][1], R0[0][2], R0[1][0], R0[1][1], R0[1][2],
                                    R0[2][0], R0[2][1], R0[2][2]};
        sphere_env<TERR, -1>(m, xw, xpw, ypw, zw, m.tsph_r, cb, T.w, T.v, toTrunk, pa_n, pa_f, on);
        if (BOX) {
            const auto tsph_pos = [&](F2& X, F2& Y, F2& Z) {
                if (TERR != 0) {
                    X = xpw;
                    Y = ypw;
                } else {
                    F2 qx[3], qy[3];
                    quat_rows01(T.quat, T.quatl, qx, qy);
                    X = f2_add(px_t, f2_mulf(qx[0], tx));
                    Y = f2_add(py_t, f2_mulf(qy[0], tx));
                }
                Z = zw;
            };
            sphere_vs_box<-1>(m, BK, Bx, xw, m.tsph_r, cb, T.w, T.v, toTrunk, pa_n, pa_f, bx_t, bx_f, tsph_pos, on);
        }
    }
    // ---- the box's 8 corner spheres against the static environment, 2 per lane
    if (BOX) {
        const TrunkFrame toBox = {BK.R[0][0], BK.R[0][1], BK.R[0][2], BK.R[1][0], BK.R[1][1], BK.R[1][2],
                                  BK.R[2][0], BK.R[2][1], BK.R[2][2]};
        const F2 bz0 = BK.rz[0], bz1 = BK.rz[1], bz2 = BK.rz[2];
#pragma unroll
        for (int cc = 0; cc < 2; cc++) {
            const int cn = 2 * leg + cc;
            const float3 cl = f3((cn & 1) ? m.box_half[0] : -m.box_half[0], (cn & 2) ? m.box_half[1] : -m.box_half[1],
                                 (cn & 4) ? m.box_half[2] : -m.box_half[2]);
            const float3 xc = BK.p + mulR(BK.R, cl);
            const F2 zc = f2_add(F2{Bx.p[2], Bx.pl[2]},
                                 f2_add(f2_mulf(bz0, cl.x), f2_add(f2_mulf(bz1, cl.y), f2_mulf(bz2, cl.z))));
            // (the free box's corners are placed horizontally from FP32 values: the
            // box tasks run on flat ground)
            sphere_env<TERR, 1>(m, xc, F2{xc.x, 0.f}, F2{xc.y, 0.f}, zc, m.box_cr, cl, BK.w, BK.v, toBox, bx_t, bx_f);
        }
    }

    // ---- trunk: sum the 4 legs' contributions (27 values: 13 packed pairs and
    // one single), add the trunk's own terms
    float Mt[6][6], bt[6];
    float3 sn, sf;   // the legs' bias terms less the lanes' trunk-sphere wrenches, summed
    {
        float v[27];
#pragma unroll
        for (int i = 0; i < 6; i++) {
            v[i] = IA.A[i];
            v[6 + i] = IA.C[i];
        }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) v[12 + 3 * i + j] = IA.B[i][j];
        v[21] = pa_n.x; v[22] = pa_n.y; v[23] = pa_n.z;
        v[24] = pa_f.x; v[25] = pa_f.y; v[26] = pa_f.z;
#pragma unroll
        for (int q = 0; q < 13; q++) xsum4_pair(v[2 * q], v[2 * q + 1]);
        v[26] = xsum4(v[26]);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i; j < 3; j++) {
                Mt[i][j] = v[sidx(i, j)];
                Mt[3 + i][3 + j] = v[6 + sidx(i, j)];
            }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Mt[i][3 + j] = v[12 + 3 * i + j];
        sn = f3(v[21], v[22], v[23]);
        sf = f3(v[24], v[25], v[26]);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Mt[i][i] += m.tr_Ic[i];
        Mt[3 + i][3 + i] += m.tr_m;
    }
    {
        // the trunk's own bias v x* I v, once, on the summed terms
        const float3 Iw = f3(m.tr_Ic[0] * T.w.x, m.tr_Ic[1] * T.w.y, m.tr_Ic[2] * T.w.z);
        const float3 bn = cross_acc(T.w, Iw, sn);
        const float3 mv = m.tr_m * T.v;
        const float3 bf = cross_acc(T.w, mv, sf);
        bt[0] = bn.x; bt[1] = bn.y; bt[2] = bn.z;
        bt[3] = bf.x; bt[4] = bf.y; bt[5] = bf.z;
    }
    // ---- solve Mt a' = -bt by the Schur complement of the linear block:
    // Mt = [A B; B^T C], C^-1 and S^-1 (S = A - B C^-1 B^T) by 3x3 cofactors
    float a0[6];
    {
        const float C00 = Mt[3][3], C01 = Mt[3][4], C02 = Mt[3][5], C11 = Mt[4][4], C12 = Mt[4][5], C22 = Mt[5][5];
        float ci[6];
        ci[0] = C11 * C22 - C12 * C12;
        ci[1] = C02 * C12 - C01 * C22;
        ci[2] = C01 * C12 - C02 * C11;
        ci[3] = C00 * C22 - C02 * C02;
        ci[4] = C01 * C02 - C00 * C12;
        ci[5] = C00 * C11 - C01 * C01;
        const float idc = rcp_approx(C00 * ci[0] + C01 * ci[1] + C02 * ci[2]);
#pragma unroll
        for (int i = 0; i < 6; i++) ci[i] *= idc;
        // W = B C^-1 (3x3)
        float W[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                W[i][j] = Mt[i][3] * ci[sidx(0, j)] + Mt[i][4] * ci[sidx(1, j)] + Mt[i][5] * ci[sidx(2, j)];
        // S = A - W B^T (symmetric)
        float S[6];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i; j < 3; j++)
                S[sidx(i, j)] = fmaf(-W[i][0], Mt[j][3], fmaf(-W[i][1], Mt[j][4], fmaf(-W[i][2], Mt[j][5], Mt[i][j])));
        float si[6];
        si[0] = S[3] * S[5] - S[4] * S[4];
        si[1] = S[2] * S[4] - S[1] * S[5];
        si[2] = S[1] * S[4] - S[2] * S[3];
        si[3] = S[0] * S[5] - S[2] * S[2];
        si[4] = S[1] * S[2] - S[0] * S[4];
        si[5] = S[0] * S[3] - S[1] * S[1];
        const float ids = rcp_approx(S[0] * si[0] + S[1] * si[1] + S[2] * si[2]);
        // [A B; B^T C] [x; y] = -[p; q]:  x = S^-1 (-p + W q),  y = C^-1 (-q - B^T x)
        float rx[3];
#pragma unroll
        for (int i = 0; i < 3; i++) rx[i] = fmaf(W[i][0], bt[3], fmaf(W[i][1], bt[4], fmaf(W[i][2], bt[5], -bt[i])));
#pragma unroll
        for (int i = 0; i < 3; i++)
            a0[i] = ids * (si[sidx(i, 0)] * rx[0] + si[sidx(i, 1)] * rx[1] + si[sidx(i, 2)] * rx[2]);
        float ry[3];
#pragma unroll
        for (int j = 0; j < 3; j++)
            ry[j] = fmaf(-Mt[0][3 + j], a0[0], fmaf(-Mt[1][3 + j], a0[1], fmaf(-Mt[2][3 + j], a0[2], -bt[3 + j])));
#pragma unroll
        for (int j = 0; j < 3; j++)
            a0[3 + j] = ci[sidx(j, 0)] * ry[0] + ci[sidx(j, 1)] * ry[1] + ci[sidx(j, 2)] * ry[2];
    }

    // ---- pass 3 (root to tip): a' = X a'_parent + c ; qdd = (u - U . a') / D
    float qdd[3];
    const float3 aw = f3(a0[0], a0[1], a0[2]), av = f3(a0[3], a0[4], a0[5]);
    {
        float3 nw = Ex_vp(c0, s0, aw, ch_w), nv = Ex_vp(c0, s0, cross_acc(aw, rh, av), ch_v);
        qdd[0] = D0inv * fmaf(-U0a[0], nw.x, fmaf(-U0a[1], nw.y, fmaf(-U0a[2], nw.z,
                         fmaf(-U0l[0], nv.x, fmaf(-U0l[1], nv.y, fmaf(-U0l[2], nv.z, u0))))));
        nw.x += qdd[0];
        float3 tw = Ey_vp(c1, s1, nw, ct_w), tv = Ey_vp(c1, s1, cross_y_acc(nw, ty, nv), ct_v);
        qdd[1] = D1inv * fmaf(-U1a[0], tw.x, fmaf(-U1a[1], tw.y, fmaf(-U1a[2], tw.z,
                         fmaf(-U1l[0], tv.x, fmaf(-U1l[1], tv.y, fmaf(-U1l[2], tv.z, u1))))));
        tw.y += qdd[1];
        float3 kw = Ey_vp(c2, s2, tw, cc_w), kv = Ey_vp(c2, s2, cross_z_acc(tw, kz, tv), cc_v);
        qdd[2] = D2inv * fmaf(-U2a, kw.y, fmaf(-U2l, kv.x, u2));
    }

    // ---- semi-implicit Euler; the position updates' rounding errors go into the
    // compensation terms (Fast2Sum)
#pragma unroll
    for (int i = 0; i < 3; i++) {
        S.qd[i] = fmaf(h, qdd[i], S.qd[i]);
        const F2 t = fast_two_sum(S.q[i], h * S.qd[i]);
        S.q[i] = t.h;
        S.ql[i] += t.l;
    }
    // v += h (a + R0^T (0, 0, g)), hg = h g
    T.w = f3(fmaf(h, aw.x, T.w.x), fmaf(h, aw.y, T.w.y), fmaf(h, aw.z, T.w.z));
    T.v = f3(fmaf(h, av.x, fmaf(hg, R0[2][0], T.v.x)), fmaf(h, av.y, fmaf(hg, R0[2][1], T.v.y)),
             fmaf(h, av.z, fmaf(hg, R0[2][2], T.v.z)));
    const float3 dp = mulR(R0, T.v);
    advance_pos<TERR != 0 || BOX>(T.p, T.pl, dp, h);
    quat_integrate_pair(T.quat, T.quatl, T.qc, T.w, h);
    if (BOX) {
        // Newton-Euler of the box about its centre (principal axes), from the summed wrench
        float3 tb = bx_t, fb = bx_f;
        xsum4_pair(tb.x, tb.y);
        xsum4_pair(tb.z, fb.x);
        xsum4_pair(fb.y, fb.z);
        const float3 Iw = f3(m.box_Ic[0] * BK.w.x, m.box_Ic[1] * BK.w.y, m.box_Ic[2] * BK.w.z);
        const float3 wxIw = cross3(BK.w, Iw), wxv = cross3(BK.w, BK.v);
        const float3 aw_b = f3((tb.x - wxIw.x) * m.box_inv_Ic[0], (tb.y - wxIw.y) * m.box_inv_Ic[1],
                               (tb.z - wxIw.z) * m.box_inv_Ic[2]);
        const float3 gbx = f3(BK.R[2][0] * g, BK.R[2][1] * g, BK.R[2][2] * g);
        const float3 av_b = m.box_inv_m * fb - wxv + gbx;
        Bx.w = Bx.w + h * aw_b;
        Bx.v = Bx.v + h * av_b;
        const float3 dpb = mulR(BK.R, Bx.v);
        advance_pos<true>(Bx.p, Bx.pl, dpb, h);
        quat_integrate_pair(Bx.quat, Bx.quatl, Bx.qc, Bx.w, h);
    }
}


// ---------------------------------------------------------------- one rollout

// Parameters of one horizon of one instance.
struct HorizonArgs {
    int H, n_sub, nx;
    float h, dt, inv_Hm1, t0, arm;
    int interp;           // INTERP_*
    const float4* Bt;     // [H] knot weights of each dt step (knot representations)
};

// x_t of rollout k: lane 0 writes the trunk, every lane its leg's joints
template <bool BOX>
__device__ __forceinline__ void store_state(float* traj, int H, int k, int t, int leg, bool valid, const Trunk& T,
                                            const LegState& S, const BoxState& Bx, int m_nx) {
    if (!valid) return;
    float* o = traj + ((size_t)k * (H + 1) + t) * m_nx;
    if (BOX && leg == 1) {
        o[37] = Bx.p[0]; o[38] = Bx.p[1]; o[39] = Bx.p[2];
        o[40] = Bx.quat[0]; o[41] = Bx.quat[1]; o[42] = Bx.quat[2]; o[43] = Bx.quat[3];
        o[44] = Bx.w.x; o[45] = Bx.w.y; o[46] = Bx.w.z;
        o[47] = Bx.v.x; o[48] = Bx.v.y; o[49] = Bx.v.z;
    }
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
}


// The trajectory pointer through an opaque move inside the horizon loop, so that
// the compiler keeps one copy of the loop (no unswitching on traj == nullptr):
// rollouts with and without trajectory output run the same instructions and
// give bit-identical results.
__device__ __forceinline__ float* opaque_ptr(float* p) {
    float* q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

// Joint targets of this lane's leg at dt step t: the knot representation's
// weights of step t (a table computed per controller: the cubic's Lagrange
// basis, the zeroth-order or linear weights) applied to Uk, or, DIRECT, the
// step's own sampled targets (Urow = the sample's [t][12] targets).
template <bool DIRECT>
__device__ __forceinline__ void leg_controls(const HorizonArgs& a, int t, int leg, const float (&Uk)[NKNOT][3],
                                             const float* Urow, float u[3]) {
    if (DIRECT) {
        const float* ut = Urow + t * NJ + 3 * leg;
        u[0] = __ldg(ut);
        u[1] = __ldg(ut + 1);
        u[2] = __ldg(ut + 2);
        return;
    }
    const float4 b = __ldg(a.Bt + t);
#pragma unroll
    for (int i = 0; i < 3; i++) u[i] = b.x * Uk[0][i] + b.y * Uk[1][i] + b.z * Uk[2][i] + b.w * Uk[3][i];
}

// One lane's share of rollout k: x0 (state), Uk[4][3] (this leg's knots) or, for
// DIRECT, Urow (the sample's H x 12 targets), the horizon, optional trajectory
// output traj (float[n][H + 1][nx], or nullptr); returns the rollout's total cost
// on every lane of the rollout.
template <int TERR, bool BOX, bool DIRECT = false>
__device__ __forceinline__ float rollout_lane(const DevModel& m, const DevCost& c, const HorizonArgs& a,
                                              const float* x0, const float (&Uk)[NKNOT][3], const float* Urow,
                                              int leg, int k, bool valid, float* traj) {

    Trunk T;
    T.p[0] = x0[0]; T.p[1] = x0[1]; T.p[2] = x0[2];
    T.pl[0] = 0.f; T.pl[1] = 0.f; T.pl[2] = 0.f;
    T.quatl[0] = 0.f; T.quatl[1] = 0.f; T.quatl[2] = 0.f; T.quatl[3] = 0.f;
    T.quat[0] = x0[3]; T.quat[1] = x0[4]; T.quat[2] = x0[5]; T.quat[3] = x0[6];
    T.qc = quat_half_norm_err(T.quat);
    T.w = f3(x0[19], x0[20], x0[21]);
    T.v = f3(x0[22], x0[23], x0[24]);
    LegState S;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        S.q[i] = x0[7 + 3 * leg + i];
        S.qd[i] = x0[25 + 3 * leg + i];
        S.ql[i] = 0.f;
    }
    BoxState Bx;
    if (BOX) {
        Bx.p[0] = x0[37]; Bx.p[1] = x0[38]; Bx.p[2] = x0[39];
        Bx.quat[0] = x0[40]; Bx.quat[1] = x0[41]; Bx.quat[2] = x0[42]; Bx.quat[3] = x0[43];
        Bx.w = f3(x0[44], x0[45], x0[46]);
        Bx.v = f3(x0[47], x0[48], x0[49]);
    }
    Bx.pl[0] = 0.f; Bx.pl[1] = 0.f; Bx.pl[2] = 0.f;
    Bx.quatl[0] = 0.f; Bx.quatl[1] = 0.f; Bx.quatl[2] = 0.f; Bx.quatl[3] = 0.f;
    Bx.qc = 0.f;
    if (BOX) Bx.qc = quat_half_norm_err(Bx.quat);
    const float h = a.h;
    const float kdh = fmaf(m.kp, h, m.kd), hg = h * m.gz;
    const LegGeom G = leg_geom(m, leg);
    const float ph0 = (leg == 1 || leg == 2) ? 3.14159265358979f : 0.f;
    float L = 0.f;
    if (float* tp = opaque_ptr(traj)) store_state<BOX>(tp, a.H, k, 0, leg, valid, T, S, Bx, a.nx);
    for (int t = 0; t < a.H; t++) {
        float u[3];
        leg_controls<DIRECT>(a, t, leg, Uk, Urow, u);
        // stage cost: this leg's control term; the trunk terms on lane 0
        {
            float ds = 0.f, dk = 0.f;
            if (c.gait != 0) {
                float s, cq;
                sincos_r(c.two_pi_over_period * (a.t0 + (float)t * a.dt) + ph0, s, cq);
                const float sw = fmaxf(s, 0.f);
                ds = c.hip_amp * s;
                dk = -c.knee_amp * sw;
                if (c.gait == 2) {
                    // Raibert foot placement: dx ahead of the hip, as a hip-flexion rotation
                    const float vx = T.v.x;
                    const float dx = c.quarter_period * vx + c.raibert_k * (vx - c.v_ref);
                    const float dth = fminf(fmaxf(-dx * c.inv_raibert_len, -0.4f), 0.4f);
                    ds += sw * dth;
                }
            }
            float e0 = u[0] - c.stand[0], e1 = u[1] - (c.stand[1] + ds), e2 = u[2] - (c.stand[2] + dk);
            L += c.w_u * (e0 * e0 + e1 * e1 + e2 * e2);
            // every lane evaluates the trunk terms (no divergent branch), lane 0 keeps them
            const float Lt = trunk_state_cost<TERR>(m, c, T) + (BOX ? box_cost(c, Bx) : 0.f);
            L += leg == 0 ? Lt : 0.f;
        }
        const float kpu[3] = {m.kp * u[0], m.kp * u[1], m.kp * u[2]};
        for (int sb = 0; sb < a.n_sub; sb++) substep<TERR, BOX>(m, leg, G, T, S, kpu, h, kdh, hg, a.arm, Bx);
        round_state<BOX>(T, S, Bx);
        if (float* tp = opaque_ptr(traj)) store_state<BOX>(tp, a.H, k, t + 1, leg, valid, T, S, Bx, a.nx);
    }
    if (leg == 0) L += c.w_term * (trunk_state_cost<TERR>(m, c, T) + (BOX ? box_cost(c, Bx) : 0.f));
    return xsum4(L);
}

}  // namespace mppi
