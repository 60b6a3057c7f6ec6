/*
 * world.c -- quadruped model, terrain, contacts, PD tracking, semi-implicit
 * Euler sub-stepping, L_walk / L_box costs and rollouts (FP64 oracle).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper: arXiv 2409.10469.  The paper's rollouts run MuJoCo (Sec. III-A); this
 * is the project's own replacement model.  Cost: L_walk (Sec. IV-B, sum over
 * t = 0..T of state and control tracking terms with diagonal Q, R) and L_box
 * (Sec. IV-D, Q_box * l1 distance of the box to its goal).  Joint targets are a
 * cubic spline through 4 evenly spaced knots (Sec. III-B, Fig. 2) tracked by PD
 * (Sec. IV-A).
 */
#include <math.h>
#include <string.h>
#include <pthread.h>
#include <stdlib.h>
#include "oracle.h"

/* ---------------- model construction ---------------- */

static void rod_inertia(double m, double len, double rad, double Ic[9]) {
    /* uniform rod along z: I_perp = m L^2 / 12, I_axis = m r^2 / 2 */
    memset(Ic, 0, sizeof(double) * 9);
    Ic[0] = m * len * len / 12.0;
    Ic[4] = m * len * len / 12.0;
    Ic[8] = m * rad * rad / 2.0;
}

void or_world_init(or_world* w, const or_params* p) {
    memset(w, 0, sizeof(*w));
    or_tree* t = &w->tree;
    or_tree_init(t, 1, -p->gravity);
    /* trunk: solid box about its centre, frame at the centre of mass */
    double a = p->trunk_size[0], b = p->trunk_size[1], c = p->trunk_size[2], m = p->trunk_mass;
    double Itr[9] = {m * (b * b + c * c) / 12.0, 0, 0, 0, m * (a * a + c * c) / 12.0, 0,
                     0, 0, m * (a * a + b * b) / 12.0};
    double zero3[3] = {0, 0, 0};
    or_tree_add(t, -1, 0, zero3, m, zero3, Itr);
    /* legs FR, FL, RR, RL: (front +x / rear -x) x (right -y / left +y) */
    static const double fx[4] = {1, 1, -1, -1}, sy[4] = {-1, 1, -1, 1};
    int nsph = 0;
    for (int l = 0; l < 4; l++) {
        double rh[3] = {fx[l] * p->hip_x, sy[l] * p->hip_y, p->hip_z};
        double Iabd = 0.4 * p->abd_mass * p->abd_radius * p->abd_radius;
        double Ia[9] = {Iabd, 0, 0, 0, Iabd, 0, 0, 0, Iabd};
        int hip = or_tree_add(t, 0, 0, rh, p->abd_mass, zero3, Ia);
        double rt[3] = {0, sy[l] * p->thigh_offset_y, 0};
        double ct[3] = {0, 0, -0.5 * p->thigh_length}, It[9];
        rod_inertia(p->thigh_mass, p->thigh_length, p->rod_radius, It);
        int thigh = or_tree_add(t, hip, 1, rt, p->thigh_mass, ct, It);
        double rc[3] = {0, 0, -p->thigh_length};
        double cc[3] = {0, 0, -0.5 * p->calf_length}, Icf[9];
        rod_inertia(p->calf_mass, p->calf_length, p->rod_radius, Icf);
        int calf = or_tree_add(t, thigh, 1, rc, p->calf_mass, cc, Icf);
        w->sph_body[nsph] = calf;
        w->sph_pos[nsph][0] = 0; w->sph_pos[nsph][1] = 0; w->sph_pos[nsph][2] = -p->calf_length;
        w->sph_r[nsph] = p->foot_radius;
        nsph++;
    }
    for (int s = 0; s < p->n_trunk_spheres && nsph < OR_MAXS; s++) {
        w->sph_body[nsph] = 0;
        w->sph_pos[nsph][0] = p->trunk_sphere_x[s];
        w->sph_pos[nsph][1] = 0;
        w->sph_pos[nsph][2] = 0;
        w->sph_r[nsph] = p->trunk_sphere_r;
        nsph++;
    }
    w->nsph = nsph;
    w->kp = p->kp; w->kd = p->kd; w->arm0 = p->armature;
    w->k = p->k_contact; w->c = p->c_contact; w->mu = p->mu; w->eps_v = p->eps_v;
    w->has_box = p->has_box;
    if (p->has_box) {
        w->box_m = p->box_mass;
        for (int i = 0; i < 3; i++) w->box_half[i] = 0.5 * p->box_size[i];
        double X = p->box_size[0], Y = p->box_size[1], Z = p->box_size[2];
        w->box_Ic[0] = p->box_mass * (Y * Y + Z * Z) / 12.0;
        w->box_Ic[1] = p->box_mass * (X * X + Z * Z) / 12.0;
        w->box_Ic[2] = p->box_mass * (X * X + Y * Y) / 12.0;
        w->box_corner_r = p->box_corner_r;
    }
    w->terrain = p->terrain;
    w->hf_nx = p->hf_nx; w->hf_ny = p->hf_ny; w->hf_cell = p->hf_cell;
    w->hf_x0 = p->hf_x0; w->hf_y0 = p->hf_y0; w->hf = p->hf;
    w->n_sbox = p->n_static_boxes;
    for (int i = 0; i < p->n_static_boxes && i < OR_MAXSBOX; i++)
        for (int a = 0; a < 3; a++) { w->sbox_lo[i][a] = p->sbox_lo[i][a]; w->sbox_hi[i][a] = p->sbox_hi[i][a]; }
    w->nx = p->has_box ? 50 : 37;
}

int or_world_nx(const or_world* w) { return w->nx; }

/* ---------------- terrain and contact geometry ---------------- */

/* height and gradient of the terrain under (x, y): plane z = 0, or a bilinear
 * heightfield clamped at its edges (zero slope across a clamped edge) */
void or_terrain_height(const or_world* w, real x, real y, real* h, real* hx, real* hy) {
    if (w->terrain != 1) { *h = 0; *hx = 0; *hy = 0; return; }
    int nx = w->hf_nx, ny = w->hf_ny;
    real u = (x - w->hf_x0) / w->hf_cell, v = (y - w->hf_y0) / w->hf_cell;
    int inx = (u >= 0 && u <= nx - 1), iny = (v >= 0 && v <= ny - 1);
    if (u < 0) u = 0;
    if (u > nx - 1) u = nx - 1;
    if (v < 0) v = 0;
    if (v > ny - 1) v = ny - 1;
    int i = (int)floor(u), j = (int)floor(v);
    if (i > nx - 2) i = nx - 2;
    if (j > ny - 2) j = ny - 2;
    real fx = u - i, fy = v - j;
    real h00 = w->hf[j * nx + i], h10 = w->hf[j * nx + i + 1];
    real h01 = w->hf[(j + 1) * nx + i], h11 = w->hf[(j + 1) * nx + i + 1];
    *h = (1 - fx) * (1 - fy) * h00 + fx * (1 - fy) * h10 + (1 - fx) * fy * h01 + fx * fy * h11;
    *hx = inx ? ((1 - fy) * (h10 - h00) + fy * (h11 - h01)) / w->hf_cell : 0;
    *hy = iny ? ((1 - fx) * (h01 - h00) + fx * (h11 - h10)) / w->hf_cell : 0;
}

/* sphere (centre x, radius r) against an axis-aligned box [lo, hi]; returns
 * 1 with the outward normal and penetration depth when they overlap */
static int sphere_aabb(const real x[3], real r, const real lo[3], const real hi[3],
                       real n[3], real* pen) {
    real cp[3], d2 = 0;
    for (int a = 0; a < 3; a++) {
        cp[a] = x[a] < lo[a] ? lo[a] : (x[a] > hi[a] ? hi[a] : x[a]);
        d2 += (x[a] - cp[a]) * (x[a] - cp[a]);
    }
    if (d2 > 0) {
        real d = sqrt(d2);
        if (d >= r) return 0;
        for (int a = 0; a < 3; a++) n[a] = (x[a] - cp[a]) / d;
        *pen = r - d;
        return 1;
    }
    /* centre inside: leave through the nearest face (order x-lo, x-hi, y-lo, ...) */
    real best = 0; int bf = -1;
    for (int a = 0; a < 3; a++) {
        real dl = x[a] - lo[a], dh = hi[a] - x[a];
        if (bf < 0 || dl < best) { best = dl; bf = 2 * a; }
        if (dh < best) { best = dh; bf = 2 * a + 1; }
    }
    n[0] = n[1] = n[2] = 0;
    n[bf / 2] = (bf & 1) ? 1 : -1;
    *pen = r + best;
    return 1;
}

/* spring-damper normal force with regularised Coulomb friction; v = velocity of
 * the contact point, n = normal pointing out of the obstacle */
static void contact_force(const or_world* w, real pen, const real n[3], const real v[3],
                          real f[3]) {
    real vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    real fn = w->k * pen - w->c * vn;
    if (fn < 0) fn = 0;
    real vt[3], vt2 = 0;
    for (int a = 0; a < 3; a++) { vt[a] = v[a] - vn * n[a]; vt2 += vt[a] * vt[a]; }
    real s = sqrt(vt2 + w->eps_v * w->eps_v);
    for (int a = 0; a < 3; a++) f[a] = fn * n[a] - w->mu * fn * vt[a] / s;
}

/* contact candidates of a sphere with the static environment: ground (index 0)
 * then each static box.  Returns 1 if candidate idx is in contact. */
static int env_contact(const or_world* w, int idx, const real x[3], real r, real n[3], real* pen) {
    if (idx == 0) {
        real h, hx, hy;
        or_terrain_height(w, x[0], x[1], &h, &hx, &hy);
        real inv = 1.0 / sqrt(hx * hx + hy * hy + 1.0);
        n[0] = -hx * inv; n[1] = -hy * inv; n[2] = inv;
        *pen = r - (x[2] - h) * n[2];
        return *pen > 0;
    }
    return sphere_aabb(x, r, w->sbox_lo[idx - 1], w->sbox_hi[idx - 1], n, pen);
}

static void cross3(const real a[3], const real b[3], real c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* velocity (world) of the body-fixed point at world position pw */
static void point_vel(const real R[3][3], const real p[3], const real vb[6], const real pw[3],
                      real vw[3]) {
    real d[3], cb[3], vpt[3];
    for (int a = 0; a < 3; a++) d[a] = pw[a] - p[a];
    for (int a = 0; a < 3; a++) cb[a] = R[0][a] * d[0] + R[1][a] * d[1] + R[2][a] * d[2];
    cross3(vb, cb, vpt);
    for (int a = 0; a < 3; a++) vpt[a] += vb[3 + a];
    for (int a = 0; a < 3; a++) vw[a] = R[a][0] * vpt[0] + R[a][1] * vpt[1] + R[a][2] * vpt[2];
}

/* add world force f applied at world point pw to a body's spatial force (body coords) */
static void add_force(const real R[3][3], const real p[3], const real pw[3], const real f[3],
                      real fb[6]) {
    real d[3], cb[3], fl[3], m[3];
    for (int a = 0; a < 3; a++) d[a] = pw[a] - p[a];
    for (int a = 0; a < 3; a++) {
        cb[a] = R[0][a] * d[0] + R[1][a] * d[1] + R[2][a] * d[2];
        fl[a] = R[0][a] * f[0] + R[1][a] * f[1] + R[2][a] * f[2];
    }
    cross3(cb, fl, m);
    for (int a = 0; a < 3; a++) { fb[a] += m[a]; fb[3 + a] += fl[a]; }
}

/*
 * External spatial forces (body coordinates) on every robot body, and on the
 * free box (fbox, box body coordinates about its centre), from all contacts.
 * Each contact acts at the deepest point of the sphere, centre - r n, with the
 * velocity of the body-fixed point there.
 */
void or_contact_fext(const or_world* w, const real* x, real fext[][6], real fbox[6]) {
    const or_tree* t = &w->tree;
    real R[OR_MAXB][3][3], p[OR_MAXB][3], vb[OR_MAXB][6];
    int nq = or_tree_nq(t), nv = or_tree_nv(t);
    const real* q = x;
    const real* v = x + nq;
    or_fk(t, q, R, p);
    or_body_vel(t, q, v, vb);
    memset(fext, 0, sizeof(real) * 6 * t->nb);
    real Rb[3][3], pb[3], vbox[6];
    if (w->has_box) {
        const real* qb = x + nq + nv;
        or_quat_to_R(qb + 3, Rb);
        for (int a = 0; a < 3; a++) pb[a] = qb[a];
        for (int a = 0; a < 6; a++) vbox[a] = x[nq + nv + 7 + a];
        for (int a = 0; a < 6; a++) fbox[a] = 0;
    }
    for (int s = 0; s < w->nsph; s++) {
        int b = w->sph_body[s];
        real xc[3], r = w->sph_r[s];
        for (int a = 0; a < 3; a++)
            xc[a] = p[b][a] + R[b][a][0] * w->sph_pos[s][0] + R[b][a][1] * w->sph_pos[s][1] +
                    R[b][a][2] * w->sph_pos[s][2];
        for (int idx = 0; idx <= w->n_sbox; idx++) {
            real n[3], pen;
            if (!env_contact(w, idx, xc, r, n, &pen)) continue;
            real pc[3], vc[3], f[3];
            for (int a = 0; a < 3; a++) pc[a] = xc[a] - r * n[a];
            point_vel(R[b], p[b], vb[b], pc, vc);
            contact_force(w, pen, n, vc, f);
            add_force(R[b], p[b], pc, f, fext[b]);
        }
        if (w->has_box) {
            /* robot sphere against the free box (oriented box, its own frame) */
            real d[3], xl[3], lo[3], hi[3], nl[3], pen;
            for (int a = 0; a < 3; a++) d[a] = xc[a] - pb[a];
            for (int a = 0; a < 3; a++) {
                xl[a] = Rb[0][a] * d[0] + Rb[1][a] * d[1] + Rb[2][a] * d[2];
                lo[a] = -w->box_half[a]; hi[a] = w->box_half[a];
            }
            if (sphere_aabb(xl, r, lo, hi, nl, &pen)) {
                real n[3], pc[3], vc[3], vcb[3], vrel[3], f[3], fm[3];
                for (int a = 0; a < 3; a++) n[a] = Rb[a][0] * nl[0] + Rb[a][1] * nl[1] + Rb[a][2] * nl[2];
                for (int a = 0; a < 3; a++) pc[a] = xc[a] - r * n[a];
                point_vel(R[b], p[b], vb[b], pc, vc);
                point_vel(Rb, pb, vbox, pc, vcb);
                for (int a = 0; a < 3; a++) vrel[a] = vc[a] - vcb[a];
                contact_force(w, pen, n, vrel, f);
                add_force(R[b], p[b], pc, f, fext[b]);
                for (int a = 0; a < 3; a++) fm[a] = -f[a];
                add_force(Rb, pb, pc, fm, fbox);
            }
        }
    }
    if (w->has_box) {
        /* 8 corner spheres of the box against the static environment */
        for (int cnr = 0; cnr < 8; cnr++) {
            real cl[3] = {(cnr & 1) ? w->box_half[0] : -w->box_half[0],
                          (cnr & 2) ? w->box_half[1] : -w->box_half[1],
                          (cnr & 4) ? w->box_half[2] : -w->box_half[2]};
            real xc[3];
            for (int a = 0; a < 3; a++) xc[a] = pb[a] + Rb[a][0] * cl[0] + Rb[a][1] * cl[1] + Rb[a][2] * cl[2];
            for (int idx = 0; idx <= w->n_sbox; idx++) {
                real n[3], pen, pc[3], vc[3], f[3];
                if (!env_contact(w, idx, xc, w->box_corner_r, n, &pen)) continue;
                for (int a = 0; a < 3; a++) pc[a] = xc[a] - w->box_corner_r * n[a];
                point_vel(Rb, pb, vbox, pc, vc);
                contact_force(w, pen, n, vc, f);
                add_force(Rb, pb, pc, f, fbox);
            }
        }
    }
}

/* ---------------- integration ---------------- */

/* q <- q (x) exp(omega h), normalised; omega in body coordinates */
static void quat_integrate(real q[4], const real w[3], real h) {
    real wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    real th = wn * h;
    real cw = cos(0.5 * th);
    real sk = (th > 0) ? sin(0.5 * th) / wn : 0.5 * h;  /* sin(th/2)/|w| */
    real d[4] = {cw, sk * w[0], sk * w[1], sk * w[2]};
    real r[4];
    r[0] = q[0] * d[0] - q[1] * d[1] - q[2] * d[2] - q[3] * d[3];
    r[1] = q[0] * d[1] + q[1] * d[0] + q[2] * d[3] - q[3] * d[2];
    r[2] = q[0] * d[2] - q[1] * d[3] + q[2] * d[0] + q[3] * d[1];
    r[3] = q[0] * d[3] + q[1] * d[2] - q[2] * d[1] + q[3] * d[0];
    real nn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int a = 0; a < 4; a++) q[a] = r[a] / nn;
}

/* semi-implicit Euler for a free body: v += h a; p += h R(q_old) v_lin; q <- q exp(h w) */
static void integrate_free(real* q, real* v, const real* a, real h) {
    real R[3][3];
    for (int i = 0; i < 6; i++) v[i] += h * a[i];
    or_quat_to_R(q + 3, R);
    for (int i = 0; i < 3; i++) q[i] += h * (R[i][0] * v[3] + R[i][1] * v[4] + R[i][2] * v[5]);
    quat_integrate(q + 3, v, h);
}

/*
 * One sub-step of length h with joint targets u:
 *   contacts -> PD torque with implicit damping -> ABA -> semi-implicit Euler.
 * PD: tau = kp (u - q - h qd) - kd qd, with the implicit part h (kd + h kp) qdd
 * moved into the joint-space inertia as armature (plus the rotor armature a0).
 */
void or_substep(const or_world* w, real* x, const real u[OR_NJ], real h) {
    const or_tree* t = &w->tree;
    int nq = or_tree_nq(t), nv = or_tree_nv(t);
    real* q = x;
    real* v = x + nq;
    real fext[OR_MAXB][6], fbox[6];
    or_contact_fext(w, x, fext, fbox);
    real tau[OR_NJ], arm[OR_NJ], acc[6 + OR_NJ];
    for (int j = 0; j < OR_NJ; j++) {
        real qj = q[7 + j], qdj = v[6 + j];
        tau[j] = w->kp * (u[j] - qj - h * qdj) - w->kd * qdj;
        arm[j] = h * (w->kd + h * w->kp) + w->arm0;
    }
    or_aba(t, q, v, tau, fext, arm, acc);
    real abox[6];
    if (w->has_box) {
        /* Newton-Euler of the box about its centre (principal axes) */
        real* qb = x + nq + nv;
        real* vbx = x + nq + nv + 7;
        real Rb[3][3], gb[3], Iw[3];
        or_quat_to_R(qb + 3, Rb);
        for (int a = 0; a < 3; a++) gb[a] = Rb[0][a] * t->g[0] + Rb[1][a] * t->g[1] + Rb[2][a] * t->g[2];
        for (int a = 0; a < 3; a++) Iw[a] = w->box_Ic[a] * vbx[a];
        real wxIw[3], wxv[3];
        cross3(vbx, Iw, wxIw);
        cross3(vbx, vbx + 3, wxv);
        for (int a = 0; a < 3; a++) {
            abox[a] = (fbox[a] - wxIw[a]) / w->box_Ic[a];
            abox[3 + a] = fbox[3 + a] / w->box_m - wxv[a] + gb[a];
        }
    }
    /* joints: qd += h qdd ; q += h qd */
    for (int j = 0; j < OR_NJ; j++) {
        v[6 + j] += h * acc[6 + j];
        q[7 + j] += h * v[6 + j];
    }
    integrate_free(q, v, acc, h);
    if (w->has_box) integrate_free(x + nq + nv, x + nq + nv + 7, abox, h);
}

/* ---------------- spline ---------------- */

/* Lagrange cubic through 4 knots at tau_j = j / 3 (the unique cubic through 4 points) */
static void lagrange4(real tau, real B[OR_NKNOT]) {
    for (int j = 0; j < OR_NKNOT; j++) {
        real b = 1;
        for (int m = 0; m < OR_NKNOT; m++)
            if (m != j) b *= (tau - m / 3.0) / (j / 3.0 - m / 3.0);
        B[j] = b;
    }
}

/* basis weights of dt step t of an H-step horizon: tau_t = t / (H - 1) */
void or_spline_basis(int H, int t, real B[OR_NKNOT]) {
    real tau = (H > 1) ? (real)t / (real)(H - 1) : 0;
    lagrange4(tau, B);
}

/* joint targets at normalised time tau (clamped to [0, 1]); U layout [knot][joint] */
void or_spline_eval(const float* U, real tau, real u[OR_NJ]) {
    real B[OR_NKNOT];
    if (tau < 0) tau = 0;
    if (tau > 1) tau = 1;
    lagrange4(tau, B);
    for (int j = 0; j < OR_NJ; j++) {
        real s = 0;
        for (int k = 0; k < OR_NKNOT; k++) s += B[k] * U[k * OR_NJ + j];
        u[j] = s;
    }
}

/* parameters per sample: 4 knots x 12 joints, or 12 targets per dt step (direct) */
int or_param_dim(int interp, int H) { return interp == OR_INTERP_DIRECT ? OR_NJ * H : OR_D; }

/*
 * Knot weights of dt step t for the knot representations.  The knot interval of
 * step t is found in integers, j = floor(3 t / (H - 1)), so that the step at a
 * knot time belongs to that knot exactly; within it f = (3 t - j (H - 1)) / (H - 1).
 *   zeroth order: B_j = 1 (the knot at or before tau_t);
 *   linear: B_j = 1 - f, B_{j+1} = f (j <= 2);
 *   cubic: the Lagrange basis (or_spline_basis).
 */
void or_interp_basis(int interp, int H, int t, real B[OR_NKNOT]) {
    if (interp == OR_INTERP_CUBIC) {
        or_spline_basis(H, t, B);
        return;
    }
    for (int j = 0; j < OR_NKNOT; j++) B[j] = 0;
    if (H <= 1) {
        B[0] = 1;
        return;
    }
    int j = (3 * t) / (H - 1);
    if (j > 3) j = 3;
    if (interp == OR_INTERP_ZERO) {
        B[j] = 1;
        return;
    }
    if (j > 2) j = 2;
    real f = (real)(3 * t - j * (H - 1)) / (real)(H - 1);
    B[j] = 1 - f;
    B[j + 1] = f;
}

/* joint targets of dt step t: the knot representation's interpolant, or the
 * step's own sampled targets (direct; U layout [t][joint]) */
void or_controls(int interp, int H, int t, const float* U, real u[OR_NJ]) {
    if (interp == OR_INTERP_DIRECT) {
        for (int j = 0; j < OR_NJ; j++) u[j] = U[(size_t)t * OR_NJ + j];
        return;
    }
    real B[OR_NKNOT];
    or_interp_basis(interp, H, t, B);
    for (int j = 0; j < OR_NJ; j++) {
        real s = 0;
        for (int k = 0; k < OR_NKNOT; k++) s += B[k] * U[k * OR_NJ + j];
        u[j] = s;
    }
}

/* ---------------- cost ---------------- */

/*
 * control reference u_ref(t): the stand pose, an open-loop trot (diagonal pairs
 * FR+RL and FL+RR in antiphase), or (gait 2) that trot with the Raibert
 * heuristic's foot placement fed back from the trunk's forward velocity v_x
 * (Sec. IV-B cites the heuristic for the gait reference): a swinging foot is
 * placed dx = (T_stance / 2) v_x + k (v_x - v_ref) ahead of its hip, T_stance =
 * half the gait period, which the hip-flexion target realises as the small-angle
 * rotation -dx / L of the leg (L the effective leg length), clamped to 0.4 rad
 * and weighted by the swing profile max(0, sin phase).  x == NULL: v_x = v_ref.
 */
void or_gait_ref_x(const or_cost* c, real t_abs, const real* x, real uref[OR_NJ]) {
    static const double phase0[4] = {0, 1, 1, 0};
    real dth = 0;
    if (c->gait == 2) {
        real vx = x ? x[22] : (real)c->v_ref;
        real dx = 0.25 * c->gait_period * vx + c->raibert_k * (vx - c->v_ref);
        dth = -dx / c->raibert_len;
        if (dth > 0.4) dth = 0.4;
        if (dth < -0.4) dth = -0.4;
    }
    for (int l = 0; l < 4; l++) {
        real dh = 0, dk = 0;
        if (c->gait == 1 || c->gait == 2) {
            real ph = 2 * M_PI * t_abs / c->gait_period + M_PI * phase0[l];
            real s = sin(ph);
            real sw = s > 0 ? s : 0;
            dh = c->gait_hip_amp * s + sw * dth;
            dk = -c->gait_knee_amp * sw;
        }
        uref[3 * l + 0] = c->stand[0];
        uref[3 * l + 1] = c->stand[1] + dh;
        uref[3 * l + 2] = c->stand[2] + dk;
    }
}

void or_gait_ref(const or_cost* c, real t_abs, real uref[OR_NJ]) { or_gait_ref_x(c, t_abs, NULL, uref); }

/* height of the ground under (x, y): the plane or heightfield, or the top of a
 * static box whose footprint contains (x, y), whichever is higher */
real or_ground_under(const or_world* w, real x, real y) {
    real h, hx, hy;
    or_terrain_height(w, x, y, &h, &hx, &hy);
    for (int b = 0; b < w->n_sbox; b++)
        if (x >= w->sbox_lo[b][0] && x <= w->sbox_hi[b][0] && y >= w->sbox_lo[b][1] && y <= w->sbox_hi[b][1] &&
            w->sbox_hi[b][2] > h)
            h = w->sbox_hi[b][2];
    return h;
}

/* state terms of L_walk and L_box (x_ref: height, upright attitude, forward
 * velocity, xy goal; box xy goal in l1) */
static real state_cost(const or_world* w, const or_cost* c, const real* x) {
    const real* q = x;
    const real* v = x + 19;
    real L = 0;
    real dz = q[2] - c->z_ref - (c->z_rel ? or_ground_under(w, q[0], q[1]) : 0);
    L += c->w_z * dz * dz;
    /* e_rot = 2 vec(q_ref^-1 (x) q), q_ref = identity, sign chosen so w >= 0 */
    real sg = q[3] < 0 ? -1 : 1;
    real ex = 2 * sg * q[4], ey = 2 * sg * q[5], ez = 2 * sg * q[6];
    L += c->w_o * (ex * ex + ey * ey + ez * ez);
    real dv = v[3] - c->v_ref;
    L += c->w_v * dv * dv;
    real dx = q[0] - c->goal_xy[0], dy = q[1] - c->goal_xy[1];
    L += c->w_p * (dx * dx + dy * dy);
    if (w->has_box) {
        const real* qb = x + 37;
        L += c->w_box * (fabs(c->box_goal_xy[0] - qb[0]) + fabs(c->box_goal_xy[1] - qb[1]));
    }
    return L;
}

real or_stage_cost(const or_world* w, const or_cost* c, const real* x, const real* u, real t_abs) {
    real uref[OR_NJ], L = state_cost(w, c, x);
    or_gait_ref_x(c, t_abs, x, uref);
    for (int j = 0; j < OR_NJ; j++) L += c->w_u * (u[j] - uref[j]) * (u[j] - uref[j]);
    return L;
}

real or_terminal_cost(const or_world* w, const or_cost* c, const real* x) {
    return c->w_terminal * state_cost(w, c, x);
}

/*
 * One rollout (Alg. 1 inner loop): H dt-steps of n_sub sub-steps each; the
 * stage cost of step t is taken on (x_t, u_t) at the start of the step, the
 * terminal term on x_H.  traj (optional): x_0 .. x_H, (H + 1) x nx.
 */
real or_rollout_mode(const or_world* w, const or_cost* c, int interp, int H, int n_sub, real dt,
                     real t0, const real* x0, const float* U, real* traj) {
    real x[64], u[OR_NJ];
    int nx = w->nx;
    memcpy(x, x0, sizeof(real) * nx);
    if (traj) memcpy(traj, x, sizeof(real) * nx);
    real L = 0, h = dt / n_sub;
    for (int t = 0; t < H; t++) {
        or_controls(interp, H, t, U, u);
        L += or_stage_cost(w, c, x, u, t0 + t * dt);
        for (int s = 0; s < n_sub; s++) or_substep(w, x, u, h);
        if (traj) memcpy(traj + (size_t)(t + 1) * nx, x, sizeof(real) * nx);
    }
    L += or_terminal_cost(w, c, x);
    return L;
}

real or_rollout(const or_world* w, const or_cost* c, int H, int n_sub, real dt, real t0,
                const real* x0, const float* U, real* traj) {
    return or_rollout_mode(w, c, OR_INTERP_CUBIC, H, n_sub, dt, t0, x0, U, traj);
}

/* ---------------- many rollouts over host threads ---------------- */

typedef struct {
    const or_world* w; const or_cost* c; const or_mppi* m; double t0;
    const double* x0; int x0_per_sample; const float* U; int n;
    double* L; double* traj; int tid, nthreads;
} rollout_job;

static void* rollout_worker(void* arg) {
    rollout_job* j = (rollout_job*)arg;
    int nx = j->w->nx, H = j->m->H;
    real x0r[64];
    real* tr = j->traj ? (real*)malloc(sizeof(real) * (size_t)(H + 1) * nx) : NULL;
    for (int k = j->tid; k < j->n; k += j->nthreads) {
        const double* x0 = j->x0 + (j->x0_per_sample ? (size_t)k * nx : 0);
        for (int i = 0; i < nx; i++) x0r[i] = (real)x0[i];
        j->L[k] = (double)or_rollout_mode(j->w, j->c, j->m->interp, H, j->m->n_sub, (real)j->m->dt,
                                          (real)j->t0, x0r,
                                          j->U + (size_t)k * or_param_dim(j->m->interp, H), tr);
        if (tr)
            for (size_t i = 0; i < (size_t)(H + 1) * nx; i++)
                j->traj[(size_t)k * (H + 1) * nx + i] = (double)tr[i];
    }
    free(tr);
    return NULL;
}

void or_rollouts(const or_world* w, const or_cost* c, const or_mppi* m, double t0,
                 const double* x0, int x0_per_sample, const float* U, int n,
                 double* L_out, double* traj, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    rollout_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) {
        rollout_job jb = {w, c, m, t0, x0, x0_per_sample, U, n, L_out, traj, i, nthreads};
        jobs[i] = jb;
    }
    if (nthreads == 1) { rollout_worker(&jobs[0]); return; }
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, rollout_worker, &jobs[i]);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
}

/* ---------------- batched helpers for the parity harness ---------------- */

typedef struct {
    const or_world* w; const double* X; const double* Ut; long m; int n_sub; double h;
    double* out; int tid, nthreads;
} dtstep_job;

static void* dtstep_worker(void* arg) {
    dtstep_job* j = (dtstep_job*)arg;
    int nx = j->w->nx;
    real x[64], u[OR_NJ];
    for (long i = j->tid; i < j->m; i += j->nthreads) {
        for (int a = 0; a < nx; a++) x[a] = (real)j->X[i * nx + a];
        for (int a = 0; a < OR_NJ; a++) u[a] = (real)j->Ut[i * OR_NJ + a];
        for (int s = 0; s < j->n_sub; s++) or_substep(j->w, x, u, (real)j->h);
        for (int a = 0; a < nx; a++) j->out[i * nx + a] = (double)x[a];
    }
    return NULL;
}

/* m independent dt steps (n_sub sub-steps of h) from states X[m][nx] with
 * targets Ut[m][12]; out[m][nx] */
void or_dt_steps(const or_world* w, const double* X, const double* Ut, long m, int n_sub,
                 double h, double* out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    dtstep_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) {
        dtstep_job jb = {w, X, Ut, m, n_sub, h, out, i, nthreads};
        jobs[i] = jb;
    }
    if (nthreads == 1) { dtstep_worker(&jobs[0]); return; }
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, dtstep_worker, &jobs[i]);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
}

/* stage costs of m (state, targets, time) triples, or terminal costs when t_abs is NULL */
void or_stage_costs(const or_world* w, const or_cost* c, const double* X, const double* Ut,
                    const double* t_abs, long m, double* out) {
    int nx = w->nx;
    real x[64], u[OR_NJ];
    for (long i = 0; i < m; i++) {
        for (int a = 0; a < nx; a++) x[a] = (real)X[i * nx + a];
        if (t_abs) {
            for (int a = 0; a < OR_NJ; a++) u[a] = (real)Ut[i * OR_NJ + a];
            out[i] = (double)or_stage_cost(w, c, x, u, (real)t_abs[i]);
        } else {
            out[i] = (double)or_terminal_cost(w, c, x);
        }
    }
}
