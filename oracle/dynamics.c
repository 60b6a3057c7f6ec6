/*
 * dynamics.c -- spatial algebra and rigid-body-tree algorithms (FP64 oracle).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Replaces the MuJoCo rollouts of Sec. III-A of arXiv 2409.10469 with the
 * project's own model.  Written in plain 6x6 matrix form, following
 * Featherstone, "Rigid Body Dynamics Algorithms" (2008):
 *   ABA  (articulated-body algorithm, floating base via the a' = a - a_g trick),
 *   RNEA (recursive Newton-Euler inverse dynamics),
 *   CRBA (composite-rigid-body joint-space inertia).
 * ABA is the algorithm under test; RNEA and CRBA exist to pin it.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

/* ---------------- spatial algebra ---------------- */

void or_skew(const real a[3], real S[3][3]) {
    S[0][0] = 0;     S[0][1] = -a[2]; S[0][2] = a[1];
    S[1][0] = a[2];  S[1][1] = 0;     S[1][2] = -a[0];
    S[2][0] = -a[1]; S[2][1] = a[0];  S[2][2] = 0;
}

/* motion cross product matrix: crm(v) = [w x, 0; v x, w x] */
void or_crm(const real v[6], real M[6][6]) {
    real W[3][3], V[3][3];
    or_skew(v, W);
    or_skew(v + 3, V);
    memset(M, 0, sizeof(real) * 36);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            M[i][j] = W[i][j];
            M[i + 3][j + 3] = W[i][j];
            M[i + 3][j] = V[i][j];
        }
}

/* force cross product matrix: crf(v) = -crm(v)^T */
void or_crf(const real v[6], real M[6][6]) {
    real C[6][6];
    or_crm(v, C);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) M[i][j] = -C[j][i];
}

/* spatial inertia about the frame origin of a body of mass m, centre of mass c,
 * rotational inertia Ic about the centre of mass: [Ic + m cx cx^T, m cx; m cx^T, m 1] */
void or_mcI(real m, const real c[3], const real Ic[3][3], real I[6][6]) {
    real C[3][3];
    or_skew(c, C);
    memset(I, 0, sizeof(real) * 36);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            real cct = 0;
            for (int k = 0; k < 3; k++) cct += C[i][k] * C[j][k];
            I[i][j] = Ic[i][j] + m * cct;
            I[i][j + 3] = m * C[i][j];
            I[i + 3][j] = m * C[j][i];
        }
    for (int i = 0; i < 3; i++) I[i + 3][i + 3] = m;
}

/* coordinate transform (parent -> child coordinates) of a frame rotated by +th
 * about a coordinate axis: E = R_axis(th)^T */
void or_rot_axis(int axis, real th, real E[3][3]) {
    real c = cos(th), s = sin(th);
    memset(E, 0, sizeof(real) * 9);
    if (axis == 0) {
        E[0][0] = 1; E[1][1] = c; E[1][2] = s; E[2][1] = -s; E[2][2] = c;
    } else if (axis == 1) {
        E[1][1] = 1; E[0][0] = c; E[0][2] = -s; E[2][0] = s; E[2][2] = c;
    } else {
        E[2][2] = 1; E[0][0] = c; E[0][1] = s; E[1][0] = -s; E[1][1] = c;
    }
}

/* Plucker motion transform B_X_A = [E, 0; -E rx, E], E rotates A -> B
 * coordinates, r = origin of B expressed in A */
void or_xform(const real E[3][3], const real r[3], real X[6][6]) {
    real Rx[3][3];
    or_skew(r, Rx);
    memset(X, 0, sizeof(real) * 36);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            real erx = 0;
            for (int k = 0; k < 3; k++) erx += E[i][k] * Rx[k][j];
            X[i][j] = E[i][j];
            X[i + 3][j + 3] = E[i][j];
            X[i + 3][j] = -erx;
        }
}

/* rotation matrix (body -> world) of a unit quaternion (w, x, y, z) */
void or_quat_to_R(const real q[4], real R[3][3]) {
    real w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static void mv6(const real A[6][6], const real x[6], real y[6]) {
    for (int i = 0; i < 6; i++) {
        real s = 0;
        for (int j = 0; j < 6; j++) s += A[i][j] * x[j];
        y[i] = s;
    }
}
static void mtv6(const real A[6][6], const real x[6], real y[6]) {
    for (int i = 0; i < 6; i++) {
        real s = 0;
        for (int j = 0; j < 6; j++) s += A[j][i] * x[j];
        y[i] = s;
    }
}
static void mm6(const real A[6][6], const real B[6][6], real C[6][6]) {
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            real s = 0;
            for (int k = 0; k < 6; k++) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}
/* C = X^T A X */
static void congruence(const real X[6][6], const real A[6][6], real C[6][6]) {
    real AX[6][6];
    mm6(A, X, AX);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            real s = 0;
            for (int k = 0; k < 6; k++) s += X[k][i] * AX[k][j];
            C[i][j] = s;
        }
}
static void mv3(const real A[3][3], const real x[3], real y[3]) {
    for (int i = 0; i < 3; i++) y[i] = A[i][0] * x[0] + A[i][1] * x[1] + A[i][2] * x[2];
}
static void mtv3(const real A[3][3], const real x[3], real y[3]) {
    for (int i = 0; i < 3; i++) y[i] = A[0][i] * x[0] + A[1][i] * x[1] + A[2][i] * x[2];
}

/* solve A x = b (n x n, row-major), Gaussian elimination with partial pivoting */
static int solve_dense(int n, real* A, real* b) {
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; k++) {
                real t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            }
            real t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            real f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        real s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* ---------------- tree ---------------- */

void or_tree_init(or_tree* t, int floating, double gz) {
    memset(t, 0, sizeof(*t));
    t->floating = floating;
    t->g[0] = 0; t->g[1] = 0; t->g[2] = gz;
}

int or_tree_add(or_tree* t, int parent, int axis, const double xtree[3], double mass,
                const double com[3], const double Ic[9]) {
    if (t->nb >= OR_MAXB) return -1;
    int i = t->nb++;
    real c[3] = {com[0], com[1], com[2]};
    real I3[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) I3[a][b] = Ic[a * 3 + b];
    t->parent[i] = parent;
    t->axis[i] = axis;
    for (int a = 0; a < 3; a++) t->xtree[i][a] = xtree[a];
    or_mcI(mass, c, I3, t->I[i]);
    return i;
}

static int first_jointed(const or_tree* t) { return t->floating ? 1 : 0; }
int or_tree_nq(const or_tree* t) { return t->floating ? 7 + t->nb - 1 : t->nb; }
int or_tree_nv(const or_tree* t) { return t->floating ? 6 + t->nb - 1 : t->nb; }
/* index of joint i's angle in q and its rate in v */
static int qi(const or_tree* t, int i) { return t->floating ? 7 + i - 1 : i; }
static int vi(const or_tree* t, int i) { return t->floating ? 6 + i - 1 : i; }

/* i_X_parent(i) for jointed body i */
static void joint_X(const or_tree* t, const real* q, int i, real X[6][6]) {
    real E[3][3];
    or_rot_axis(t->axis[i], q[qi(t, i)], E);
    or_xform(E, t->xtree[i], X);
}

/* world pose of every body: R[i] (body -> world), p[i] (origin, world) */
void or_fk(const or_tree* t, const real* q, real R[][3][3], real p[][3]) {
    for (int i = 0; i < t->nb; i++) {
        if (i == 0 && t->floating) {
            or_quat_to_R(q + 3, R[0]);
            for (int a = 0; a < 3; a++) p[0][a] = q[a];
            continue;
        }
        real E[3][3], Rl[3][3], pl[3];
        or_rot_axis(t->axis[i], q[qi(t, i)], E);
        int l = t->parent[i];
        if (l < 0) {
            memset(Rl, 0, sizeof(Rl));
            Rl[0][0] = Rl[1][1] = Rl[2][2] = 1;
            pl[0] = pl[1] = pl[2] = 0;
        } else {
            memcpy(Rl, R[l], sizeof(Rl));
            memcpy(pl, p[l], sizeof(pl));
        }
        /* R_i = R_l E^T ; p_i = p_l + R_l xtree */
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                real s = 0;
                for (int k = 0; k < 3; k++) s += Rl[a][k] * E[b][k];
                R[i][a][b] = s;
            }
        real d[3];
        mv3(Rl, t->xtree[i], d);
        for (int a = 0; a < 3; a++) p[i][a] = pl[a] + d[a];
    }
}

/* spatial velocity of every body in its own coordinates */
void or_body_vel(const or_tree* t, const real* q, const real* v, real vb[][6]) {
    for (int i = 0; i < t->nb; i++) {
        if (i == 0 && t->floating) {
            for (int a = 0; a < 6; a++) vb[0][a] = v[a];
            continue;
        }
        real X[6][6], vp[6] = {0, 0, 0, 0, 0, 0};
        joint_X(t, q, i, X);
        if (t->parent[i] >= 0) mv6(X, vb[t->parent[i]], vp);
        for (int a = 0; a < 6; a++) vb[i][a] = vp[a];
        vb[i][t->axis[i]] += v[vi(t, i)];
    }
}

/* gravity expressed in the coordinates of body 0 (floating) or the world */
static void base_gravity(const or_tree* t, const real* q, real ag[6]) {
    for (int a = 0; a < 6; a++) ag[a] = 0;
    if (t->floating) {
        real R[3][3];
        or_quat_to_R(q + 3, R);
        mtv3(R, t->g, ag + 3);
    } else {
        for (int a = 0; a < 3; a++) ag[3 + a] = t->g[a];
    }
}

/*
 * Articulated-body algorithm.
 *   tau[j]  : joint torques (length nb - floating)
 *   fext[i] : external spatial force on body i, body coordinates (may be NULL)
 *   arm[j]  : added joint-space inertia (implicit-PD armature), may be NULL
 *   acc     : output, length nv.  Floating: acc[0..5] = spatial acceleration of
 *             body 0 in body coordinates (d/dt of v[0..5]), then joint qdd.
 */
void or_aba(const or_tree* t, const real* q, const real* v, const real* tau,
            const real fext[][6], const real* arm, real* acc) {
    int nb = t->nb, f0 = first_jointed(t);
    real X[OR_MAXB][6][6], vb[OR_MAXB][6], c[OR_MAXB][6];
    real IA[OR_MAXB][6][6], pA[OR_MAXB][6];
    real U[OR_MAXB][6], D[OR_MAXB], u[OR_MAXB], ap[OR_MAXB][6];

    /* pass 1: velocities, velocity-product accelerations, bias forces */
    for (int i = 0; i < nb; i++) {
        real Iv[6], F[6][6];
        if (i == 0 && t->floating) {
            for (int a = 0; a < 6; a++) { vb[0][a] = v[a]; c[0][a] = 0; }
        } else {
            real vp[6] = {0, 0, 0, 0, 0, 0}, vJ[6] = {0, 0, 0, 0, 0, 0}, C[6][6];
            joint_X(t, q, i, X[i]);
            if (t->parent[i] >= 0) mv6(X[i], vb[t->parent[i]], vp);
            vJ[t->axis[i]] = v[vi(t, i)];
            for (int a = 0; a < 6; a++) vb[i][a] = vp[a] + vJ[a];
            or_crm(vb[i], C);
            mv6(C, vJ, c[i]);
        }
        memcpy(IA[i], t->I[i], sizeof(IA[i]));
        mv6(t->I[i], vb[i], Iv);
        or_crf(vb[i], F);
        mv6(F, Iv, pA[i]);
        if (fext)
            for (int a = 0; a < 6; a++) pA[i][a] -= fext[i][a];
    }
    /* pass 2: articulated inertias and bias forces, tip to root */
    for (int i = nb - 1; i >= f0; i--) {
        int k = t->axis[i], j = i - f0;
        for (int a = 0; a < 6; a++) U[i][a] = IA[i][a][k];
        D[i] = U[i][k] + (arm ? arm[j] : 0);
        u[i] = tau[j] - pA[i][k];
        int l = t->parent[i];
        if (l >= 0) {
            real Ia[6][6], pa[6], Iac[6], XIX[6][6], Xpa[6];
            for (int a = 0; a < 6; a++)
                for (int b = 0; b < 6; b++) Ia[a][b] = IA[i][a][b] - U[i][a] * U[i][b] / D[i];
            mv6(Ia, c[i], Iac);
            for (int a = 0; a < 6; a++) pa[a] = pA[i][a] + Iac[a] + U[i][a] * u[i] / D[i];
            congruence(X[i], Ia, XIX);
            mtv6(X[i], pa, Xpa);
            for (int a = 0; a < 6; a++) {
                for (int b = 0; b < 6; b++) IA[l][a][b] += XIX[a][b];
                pA[l][a] += Xpa[a];
            }
        }
    }
    /* base: a'_0 = -IA_0^-1 pA_0 (floating) or a'_world = -a_g (fixed) */
    real ag[6], aroot[6];
    base_gravity(t, q, ag);
    if (t->floating) {
        real A[36], b[6];
        for (int a = 0; a < 6; a++) {
            for (int bb = 0; bb < 6; bb++) A[a * 6 + bb] = IA[0][a][bb];
            b[a] = -pA[0][a];
        }
        solve_dense(6, A, b);
        for (int a = 0; a < 6; a++) ap[0][a] = b[a];
    }
    for (int a = 0; a < 6; a++) aroot[a] = -ag[a];
    /* pass 3: accelerations, root to tip */
    for (int i = f0; i < nb; i++) {
        int k = t->axis[i], l = t->parent[i];
        real apl[6];
        mv6(X[i], l >= 0 ? ap[l] : aroot, apl);
        for (int a = 0; a < 6; a++) ap[i][a] = apl[a] + c[i][a];
        real Ua = 0;
        for (int a = 0; a < 6; a++) Ua += U[i][a] * ap[i][a];
        real qdd = (u[i] - Ua) / D[i];
        ap[i][k] += qdd;
        acc[vi(t, i)] = qdd;
    }
    if (t->floating)
        for (int a = 0; a < 6; a++) acc[a] = ap[0][a] + ag[a];
}

/*
 * Recursive Newton-Euler inverse dynamics.  acc as produced by or_aba.
 * tau_out (length nv): floating: [net base wrench that would be needed (6), joint
 * torques]; a consistent free-floating motion gives a zero base wrench.
 */
void or_rnea(const or_tree* t, const real* q, const real* v, const real* acc,
             const real fext[][6], const real* arm, real* tau_out) {
    int nb = t->nb, f0 = first_jointed(t);
    real X[OR_MAXB][6][6], vb[OR_MAXB][6], ab[OR_MAXB][6], f[OR_MAXB][6];
    real ag[6], aroot[6];
    base_gravity(t, q, ag);
    for (int a = 0; a < 6; a++) aroot[a] = -ag[a];
    for (int i = 0; i < nb; i++) {
        if (i == 0 && t->floating) {
            for (int a = 0; a < 6; a++) { vb[0][a] = v[a]; ab[0][a] = acc[a] - ag[a]; }
        } else {
            real vp[6] = {0, 0, 0, 0, 0, 0}, apar[6], vJ[6] = {0, 0, 0, 0, 0, 0}, C[6][6], cJ[6];
            int l = t->parent[i];
            joint_X(t, q, i, X[i]);
            if (l >= 0) mv6(X[i], vb[l], vp);
            mv6(X[i], l >= 0 ? ab[l] : aroot, apar);
            vJ[t->axis[i]] = v[vi(t, i)];
            for (int a = 0; a < 6; a++) vb[i][a] = vp[a] + vJ[a];
            or_crm(vb[i], C);
            mv6(C, vJ, cJ);
            for (int a = 0; a < 6; a++) ab[i][a] = apar[a] + cJ[a];
            ab[i][t->axis[i]] += acc[vi(t, i)];
        }
        real Ia[6], Iv[6], F[6][6], bias[6];
        mv6(t->I[i], ab[i], Ia);
        mv6(t->I[i], vb[i], Iv);
        or_crf(vb[i], F);
        mv6(F, Iv, bias);
        for (int a = 0; a < 6; a++) f[i][a] = Ia[a] + bias[a] - (fext ? fext[i][a] : 0);
    }
    for (int i = nb - 1; i >= f0; i--) {
        int j = i - f0;
        tau_out[vi(t, i)] = f[i][t->axis[i]] + (arm ? arm[j] * acc[vi(t, i)] : 0);
        int l = t->parent[i];
        if (l >= 0) {
            real Xf[6];
            mtv6(X[i], f[i], Xf);
            for (int a = 0; a < 6; a++) f[l][a] += Xf[a];
        }
    }
    if (t->floating)
        for (int a = 0; a < 6; a++) tau_out[a] = f[0][a];
}

/*
 * Composite-rigid-body algorithm: joint-space inertia M (nv x nv, row-major),
 * in the same coordinates as or_aba's acc, plus diag(arm) on the joints.
 */
void or_crba(const or_tree* t, const real* q, const real* arm, real* M) {
    int nb = t->nb, nv = or_tree_nv(t), f0 = first_jointed(t);
    real X[OR_MAXB][6][6], IC[OR_MAXB][6][6];
    memset(M, 0, sizeof(real) * nv * nv);
    for (int i = 0; i < nb; i++) {
        memcpy(IC[i], t->I[i], sizeof(IC[i]));
        if (i >= f0) joint_X(t, q, i, X[i]);
    }
    for (int i = nb - 1; i >= f0; i--) {
        int l = t->parent[i];
        if (l >= 0) {
            real XIX[6][6];
            congruence(X[i], IC[i], XIX);
            for (int a = 0; a < 6; a++)
                for (int b = 0; b < 6; b++) IC[l][a][b] += XIX[a][b];
        }
    }
    if (t->floating)
        for (int a = 0; a < 6; a++)
            for (int b = 0; b < 6; b++) M[a * nv + b] = IC[0][a][b];
    for (int i = f0; i < nb; i++) {
        real F[6];
        int k = t->axis[i], ri = vi(t, i);
        for (int a = 0; a < 6; a++) F[a] = IC[i][a][k];
        M[ri * nv + ri] = F[k] + (arm ? arm[i - f0] : 0);
        int j = i;
        while (t->parent[j] >= 0) {
            real Fp[6];
            mtv6(X[j], F, Fp);
            memcpy(F, Fp, sizeof(F));
            j = t->parent[j];
            if (j == 0 && t->floating) {
                for (int a = 0; a < 6; a++) { M[a * nv + ri] = F[a]; M[ri * nv + a] = F[a]; }
            } else {
                int rj = vi(t, j);
                M[ri * nv + rj] = F[t->axis[j]];
                M[rj * nv + ri] = F[t->axis[j]];
            }
        }
    }
}

/* world-frame spatial transform of a force from body coordinates: f_w = (0_X_i)^* f_b */
static void force_to_world(const real R[3][3], const real p[3], const real fb[6], real fw[6]) {
    real n[3], f[3], pxf[3];
    mv3(R, fb, n);
    mv3(R, fb + 3, f);
    pxf[0] = p[1] * f[2] - p[2] * f[1];
    pxf[1] = p[2] * f[0] - p[0] * f[2];
    pxf[2] = p[0] * f[1] - p[1] * f[0];
    for (int a = 0; a < 3; a++) { fw[a] = n[a] + pxf[a]; fw[3 + a] = f[a]; }
}

/* total spatial momentum in world coordinates (about the world origin) */
void or_momentum_world(const or_tree* t, const real* q, const real* v, real h[6]) {
    real R[OR_MAXB][3][3], p[OR_MAXB][3], vb[OR_MAXB][6];
    or_fk(t, q, R, p);
    or_body_vel(t, q, v, vb);
    for (int a = 0; a < 6; a++) h[a] = 0;
    for (int i = 0; i < t->nb; i++) {
        real hb[6], hw[6];
        mv6(t->I[i], vb[i], hb);
        force_to_world(R[i], p[i], hb, hw);
        for (int a = 0; a < 6; a++) h[a] += hw[a];
    }
}

/* d/dt of the total spatial momentum implied by acc (true accelerations):
 * sum_i 0_X_i^* (I_i a_i + v_i x* I_i v_i).  Equals the sum of external
 * forces (world coordinates), including gravity. */
void or_momentum_rate_world(const or_tree* t, const real* q, const real* v, const real* acc,
                            real hdot[6]) {
    int nb = t->nb;
    real R[OR_MAXB][3][3], p[OR_MAXB][3], vb[OR_MAXB][6], ab[OR_MAXB][6];
    or_fk(t, q, R, p);
    for (int a = 0; a < 6; a++) hdot[a] = 0;
    for (int i = 0; i < nb; i++) {
        if (i == 0 && t->floating) {
            for (int a = 0; a < 6; a++) { vb[0][a] = v[a]; ab[0][a] = acc[a]; }
        } else {
            real X[6][6], vp[6] = {0, 0, 0, 0, 0, 0}, apar[6] = {0, 0, 0, 0, 0, 0};
            real vJ[6] = {0, 0, 0, 0, 0, 0}, C[6][6], cJ[6];
            int l = t->parent[i];
            joint_X(t, q, i, X);
            if (l >= 0) { mv6(X, vb[l], vp); mv6(X, ab[l], apar); }
            vJ[t->axis[i]] = v[vi(t, i)];
            for (int a = 0; a < 6; a++) vb[i][a] = vp[a] + vJ[a];
            or_crm(vb[i], C);
            mv6(C, vJ, cJ);
            for (int a = 0; a < 6; a++) ab[i][a] = apar[a] + cJ[a];
            ab[i][t->axis[i]] += acc[vi(t, i)];
        }
        real Ia[6], Iv[6], F[6][6], bias[6], fb[6], fw[6];
        mv6(t->I[i], ab[i], Ia);
        mv6(t->I[i], vb[i], Iv);
        or_crf(vb[i], F);
        mv6(F, Iv, bias);
        for (int a = 0; a < 6; a++) fb[a] = Ia[a] + bias[a];
        force_to_world(R[i], p[i], fb, fw);
        for (int a = 0; a < 6; a++) hdot[a] += fw[a];
    }
}
