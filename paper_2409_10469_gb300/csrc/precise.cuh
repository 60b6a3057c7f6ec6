// precise.cuh -- extended-precision pieces of the FP32 rollout arithmetic.
//
// The contact model's normal force is k pen with k = 2e4 N/m, and a sphere's
// penetration is the difference of two ~0.3 m terms (trunk height and the leg's
// vertical extent).  Plain FP32 puts ~3e-8 m of rounding on that difference,
// which k turns into ~1e-3 N and the one-step joint rates into ~1e-4 relative
// error.  So the sphere heights are evaluated as pairs hi + lo of FP32 numbers
// (error-free products by FMA, Knuth's TwoSum for sums: about 2^-44 relative),
// from joint angles and trunk positions that carry their own FP32 compensation
// term within a dt step, and sines and cosines of those angles that are
// accurate to ~1e-9: a table of sin / cos at 512 points per turn, each stored
// as an FP32 pair rounded from double precision, and a third-order Taylor step
// from the nearest point (|d| <= pi / 512), whose FP32 evaluation error stays
// below 5e-10.  Everything else in the sub-step stays plain FP32.
#pragma once
#include <cuda_runtime.h>

#include "trig_table.inc"  // g_trig[TRIG_N]: (cos_hi, cos_lo, sin_hi, sin_lo) at j 2 pi / TRIG_N (build-generated)

namespace mppi {

// a value hi + lo held as two FP32 numbers.  lo is either a correction of a few
// ulp of hi or, for the sines and cosines, the table's low part plus the Taylor
// term (below 7e-3): the pairs are not renormalised, so products keep the
// lo * lo term and sums add the low parts in FP32 (their rounding stays below
// 5e-10 at that size)
struct F2 {
    float h, l;
};

// The operations below are written with the _rn intrinsics, which the compiler
// never contracts into a fused multiply-add: a product rounded by itself and then
// fused into the next addition would break the error-free transformations.

// a + b as an exact pair (Knuth's TwoSum: no ordering assumption)
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// a + b as a pair by Dekker's Fast2Sum: exact when |a| >= |b|.  Used for a
// position plus its sub-step increment; where the increment is the larger (an
// angle within a few hundredths of zero), the error term is still within an ulp
// of the sum, and the ulp of so small a sum is far below the target precision
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a * b as an exact pair (the FMA recovers the product's rounding error)
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return s;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    F2 s = two_sum(a.h, -b.h);
    s.l = __fadd_rn(s.l, __fsub_rn(a.l, b.l));
    return s;
}
__device__ __forceinline__ F2 f2_addf(F2 a, float b) {
    F2 s = two_sum(a.h, b);
    s.l = __fadd_rn(s.l, a.l);
    return s;
}
// (a.h + a.l) (b.h + b.l): the product of the heads as an exact pair, the cross
// terms and a.l b.l into the low part
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    return {p, __fmaf_rn(a.l, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.h, b.h, -p))))};
}
// (a.h + a.l) c for an FP32 constant c
__device__ __forceinline__ F2 f2_mulf(F2 a, float c) {
    const float p = __fmul_rn(a.h, c);
    return {p, __fmaf_rn(a.l, c, __fmaf_rn(a.h, c, -p))};
}
__device__ __forceinline__ float f2_val(F2 a) { return __fadd_rn(a.h, a.l); }

// 2 pi / TRIG_N split into a 12-bit head (j * head is exact for |j| < 2^12, i.e.
// angles below 50 rad) and the rest
constexpr float TRIG_STEP_HI = 0.012271881103515625f;
constexpr float TRIG_STEP_LO = -3.480043049564063e-08f;
constexpr float TRIG_INV_STEP = 81.4873275756836f;

// sin and cos of the angle xh + xl (|xl| a few ulp of xh): the nearest table
// point a_j = j 2 pi / TRIG_N, d = x - a_j (the head's product is exact, so
// xh - j head is exact), and
//   sin(a_j + d) = S + (C d - S d^2/2 - C d^3/6),
//   cos(a_j + d) = C - (S d + C d^2/2 - S d^3/6),
// with |d| <= pi / TRIG_N (the dropped d^4/24, d^5/120 terms are below 1e-10).
// Returned as pairs (table value, its low part plus the Taylor term).
// The table in shared memory: every kernel that runs sub-steps copies it there
// once at its start (trig_to_shared, which synchronises the block), so each
// table read on the sub-step's dependency chain is a shared load rather than
// an L1 hit.
__shared__ float4 s_trig[TRIG_N];
__device__ __forceinline__ void trig_to_shared() {
    for (int i = threadIdx.x; i < TRIG_N; i += blockDim.x) s_trig[i] = g_trig[i];
    __syncthreads();
}

__device__ __forceinline__ void sincos_pair(float xh, float xl, F2& s, F2& c) {
    // the nearest table point j = rint(xh / step) by the 1.5 * 2^23 shift (|xh / step| < 2^22):
    // one FMA and one subtraction, no conversion instructions; the low bits of the
    // shifted value are j modulo the table size
    const float y = __fmaf_rn(xh, TRIG_INV_STEP, 12582912.0f);
    const float jf = __fsub_rn(y, 12582912.0f);
    const int j = __float_as_int(y) & (TRIG_N - 1);
    const float t = __fmaf_rn(-jf, TRIG_STEP_HI, xh);
    const float d = __fadd_rn(t, __fmaf_rn(-jf, TRIG_STEP_LO, xl));
    const float4 T = s_trig[j];  // cos hi, cos lo, sin hi, sin lo
    const float hd2 = __fmul_rn(0.5f, __fmul_rn(d, d));
    const float d3 = __fmul_rn(__fmul_rn(hd2, d), 1.f / 3.f);
    s.h = T.z;
    s.l = __fadd_rn(T.w, __fmaf_rn(T.x, d, -__fmaf_rn(T.z, hd2, __fmul_rn(T.x, d3))));
    c.h = T.x;
    c.l = __fsub_rn(T.y, __fmaf_rn(T.z, d, __fmaf_rn(T.x, hd2, -__fmul_rn(T.z, d3))));
}

// Row 2 of the rotation (body -> world) of the quaternion (w, x, y, z) + (lo
// parts ql) -- the world's vertical in body coordinates -- as pairs:
// (2 (x z - w y), 2 (y z + w x), 1 - 2 (x^2 + y^2)), the products of the heads
// exact, the lo parts to first order (their squares are below 2^-46).
__device__ __forceinline__ void quat_row2(const float q[4], const float ql[4], F2& r0, F2& r1, F2& r2) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float wl = ql[0], xl = ql[1], yl = ql[2], zl = ql[3];
    const F2 a = f2_sub(two_prod(x + x, z), two_prod(w + w, y));
    const F2 b = f2_add(two_prod(y + y, z), two_prod(w + w, x));
    const F2 c = f2_add(two_prod(x + x, x), two_prod(y + y, y));
    r0 = a;
    r0.l = __fmaf_rn(2.f, __fmaf_rn(xl, z, __fmaf_rn(x, zl, -__fmaf_rn(wl, y, __fmul_rn(w, yl)))), r0.l);
    r1 = b;
    r1.l = __fmaf_rn(2.f, __fmaf_rn(yl, z, __fmaf_rn(y, zl, __fmaf_rn(wl, x, __fmul_rn(w, xl)))), r1.l);
    r2 = two_sum(1.f, -c.h);
    r2.l = __fsub_rn(r2.l, __fmaf_rn(4.f, __fmaf_rn(x, xl, __fmul_rn(y, yl)), c.l));
}

// Rows 0 and 1 of the rotation (body -> world) of the quaternion q + ql as pairs
// (the world's x and y axes in body coordinates), as quat_row2:
// row 0 = (1 - 2 (y^2 + z^2), 2 (x y - w z), 2 (x z + w y)),
// row 1 = (2 (x y + w z), 1 - 2 (x^2 + z^2), 2 (y z - w x)).
__device__ __forceinline__ void quat_rows01(const float q[4], const float ql[4], F2 r0[3], F2 r1[3]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float wl = ql[0], xl = ql[1], yl = ql[2], zl = ql[3];
    const F2 yy_zz = f2_add(two_prod(y + y, y), two_prod(z + z, z));
    r0[0] = two_sum(1.f, -yy_zz.h);
    r0[0].l = __fsub_rn(r0[0].l, __fmaf_rn(4.f, __fmaf_rn(y, yl, __fmul_rn(z, zl)), yy_zz.l));
    r0[1] = f2_sub(two_prod(x + x, y), two_prod(w + w, z));
    r0[1].l = __fmaf_rn(2.f, __fmaf_rn(xl, y, __fmaf_rn(x, yl, -__fmaf_rn(wl, z, __fmul_rn(w, zl)))), r0[1].l);
    r0[2] = f2_add(two_prod(x + x, z), two_prod(w + w, y));
    r0[2].l = __fmaf_rn(2.f, __fmaf_rn(xl, z, __fmaf_rn(x, zl, __fmaf_rn(wl, y, __fmul_rn(w, yl)))), r0[2].l);
    r1[0] = f2_add(two_prod(x + x, y), two_prod(w + w, z));
    r1[0].l = __fmaf_rn(2.f, __fmaf_rn(xl, y, __fmaf_rn(x, yl, __fmaf_rn(wl, z, __fmul_rn(w, zl)))), r1[0].l);
    const F2 xx_zz = f2_add(two_prod(x + x, x), two_prod(z + z, z));
    r1[1] = two_sum(1.f, -xx_zz.h);
    r1[1].l = __fsub_rn(r1[1].l, __fmaf_rn(4.f, __fmaf_rn(x, xl, __fmul_rn(z, zl)), xx_zz.l));
    r1[2] = f2_sub(two_prod(y + y, z), two_prod(w + w, x));
    r1[2].l = __fmaf_rn(2.f, __fmaf_rn(yl, z, __fmaf_rn(y, zl, -__fmaf_rn(wl, x, __fmul_rn(w, xl)))), r1[2].l);
}

// a pair brought back to an FP32 value and a low part below half its ulp
__device__ __forceinline__ F2 f2_norm(F2 a) { return two_sum(a.h, a.l); }

// (|q|^2 - 1) / 2 of an FP32 quaternion, every square exact (the sum of the
// four squares as a pair, less one: s.h - 1 is exact near 1)
__device__ __forceinline__ float quat_half_norm_err(const float q[4]) {
    const F2 s = f2_add(f2_add(two_prod(q[0], q[0]), two_prod(q[1], q[1])),
                        f2_add(two_prod(q[2], q[2]), two_prod(q[3], q[3])));
    return __fmul_rn(0.5f, __fadd_rn(__fsub_rn(s.h, 1.f), s.l));
}

// q <- (q (x) exp(w h / 2)) / |q (x) exp(w h / 2)| for the quaternion q = qh + ql
// (w in body coordinates), c = (|q|^2 - 1) / 2 of the input (zero once the pair
// has been normalised).  With s = |w| h / 2, d = (cos s, sin s w / |w|) and
// |d| = 1, the step is q + (q (cos s - 1 - c) + T) to first order in c (T: the
// products with sin s w / |w|); that increment is small (~|w| h), so it is
// formed in FP32 and added to the pair by Fast2Sum.  cos s - 1 and sin s / |w|
// are power series in s^2 (truncation below 3e-10 for |w| h <= 1).
__device__ __forceinline__ void quat_integrate_pair(float qh[4], float ql[4], float& c, float3 w, float h) {
    const float hh = 0.5f * h;
    const float x = dot3(w, w) * (hh * hh);
    float pc = fmaf(x, 2.48015873e-05f, -1.38888889e-03f);
    pc = fmaf(x, pc, 4.16666667e-02f);
    pc = fmaf(x, pc, -0.5f);
    const float e = fmaf(x, pc, -c);  // cos s - 1 - c
    float ps = fmaf(x, 2.75573192e-06f, -1.98412698e-04f);
    ps = fmaf(x, ps, 8.33333333e-03f);
    ps = fmaf(x, ps, -1.66666667e-01f);
    const float sk = hh * fmaf(x, ps, 1.f);
    const float d1 = sk * w.x, d2 = sk * w.y, d3 = sk * w.z;
    const float q0 = qh[0], q1 = qh[1], q2 = qh[2], q3 = qh[3];
    const float dq[4] = {fmaf(q0, e, fmaf(-q1, d1, fmaf(-q2, d2, -q3 * d3))),
                         fmaf(q1, e, fmaf(q0, d1, fmaf(q2, d3, -q3 * d2))),
                         fmaf(q2, e, fmaf(q0, d2, fmaf(-q1, d3, q3 * d1))),
                         fmaf(q3, e, fmaf(q0, d3, fmaf(q1, d2, -q2 * d1)))};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const F2 t = fast_two_sum(qh[k], dq[k]);
        qh[k] = t.h;
        ql[k] = __fadd_rn(ql[k], t.l);
    }
    c = 0.f;
}

}  // namespace mppi
