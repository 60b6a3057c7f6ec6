/*
 * oracle.h -- FP64 CPU oracle for the whole-body MPPI hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this code: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs use it.  It shares no source with the
 * CUDA path (paper_2409_10469_gb300/csrc).
 *
 * What it computes (arXiv 2409.10469):
 *   - MPPI, Algorithm 1 (Sec. II-B): sample knots, roll out, accumulate cost,
 *     softmax weights (Eq. 1), weighted mean (Eq. 2), apply u = mu[0], shift.
 *   - Controls as a cubic spline over 4 knots (Sec. III-B, Fig. 2).
 *   - L_walk (Sec. IV-B) and L_box (Sec. IV-D) costs.
 *   - The simulator that the paper takes from MuJoCo (Sec. III-A) is replaced
 *     by the project's own model: Featherstone ABA on a floating-base tree,
 *     spring-damper penalty contacts with regularised Coulomb friction,
 *     semi-implicit Euler with n_sub sub-steps, PD tracking with implicit
 *     damping.  Every constant the paper leaves open is a model-spec reading.
 *
 * Precision: double everywhere, except the sampling step (Philox4x32-10,
 * Box-Muller, knot perturbation) whose FP32 operation sequence is part of the
 * model spec so that CPU and GPU agree bit for bit.
 *
 * Conventions:
 *   spatial vectors are [angular; linear] (Featherstone), body coordinates;
 *   world z up; quaternions (w, x, y, z), body -> world;
 *   floating base: q = [p(3), quat(4), joints], v = [omega_b(3), v_b(3), qd];
 *   the free box (when present) follows the robot: [q_box(7)], [v_box(6)].
 *   State vector x = [q_robot(19), v_robot(18), (q_box(7), v_box(6))].
 */
#ifndef MPPI_ORACLE_H
#define MPPI_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#ifndef OR_REAL
typedef double real;
#else
typedef OR_REAL real;
#endif

#define OR_MAXB 16      /* bodies in one tree */
#define OR_MAXS 16      /* contact spheres on the robot */
#define OR_MAXSBOX 4    /* static boxes in the environment */
#define OR_NJ 12        /* actuated joints of the quadruped */
#define OR_NKNOT 4      /* spline knots */
#define OR_D 48         /* knots x joints */

/* ---------------- kinematic tree (generic) ---------------- */
typedef struct {
    int nb;                     /* number of bodies */
    int floating;               /* 1: body 0 is a free 6-DoF body; 0: all bodies jointed */
    int parent[OR_MAXB];        /* parent body, -1 = world */
    int axis[OR_MAXB];          /* revolute joint axis (0 x, 1 y, 2 z) in the joint frame */
    real xtree[OR_MAXB][3];     /* joint origin in the parent frame (identity rotation at q = 0) */
    real I[OR_MAXB][6][6];      /* spatial inertia about the body-frame origin */
    real g[3];                  /* gravity, world frame */
} or_tree;

/* ---------------- raw model description (an input) ---------------- */
typedef struct {
    double trunk_mass, trunk_size[3];
    double hip_x, hip_y, hip_z;           /* abduction joint at (+-hip_x, +-hip_y, hip_z) */
    double abd_mass, abd_radius;          /* hip link: solid sphere about the joint */
    double thigh_offset_y;                /* flexion joint, lateral offset (x side sign) */
    double thigh_mass, thigh_length;
    double calf_mass, calf_length;
    double rod_radius;                    /* thigh/calf uniform rods */
    double foot_radius;
    int n_trunk_spheres; double trunk_sphere_x[4]; double trunk_sphere_r;
    double gravity;
    double kp, kd, armature;              /* PD gains, reflected rotor inertia a0 */
    double k_contact, c_contact, mu, eps_v;
    /* free box (config 4) */
    int has_box; double box_mass, box_size[3], box_corner_r;
    /* terrain */
    int terrain;                          /* 0 plane z = 0, 1 heightfield */
    int hf_nx, hf_ny; double hf_cell, hf_x0, hf_y0;
    const float* hf;                      /* heights [hf_ny][hf_nx], row = y */
    int n_static_boxes; double sbox_lo[OR_MAXSBOX][3], sbox_hi[OR_MAXSBOX][3];
} or_params;

typedef struct {
    or_tree tree;
    int nsph; int sph_body[OR_MAXS]; real sph_pos[OR_MAXS][3]; real sph_r[OR_MAXS];
    real kp, kd, arm0;
    real k, c, mu, eps_v;
    int has_box; real box_m, box_half[3], box_corner_r, box_Ic[3];
    int terrain; int hf_nx, hf_ny; real hf_cell, hf_x0, hf_y0; const float* hf;
    int n_sbox; real sbox_lo[OR_MAXSBOX][3], sbox_hi[OR_MAXSBOX][3];
    int nx;                     /* state size: 37, or 50 with the box */
} or_world;

/* ---------------- cost (L_walk, L_box) ---------------- */
typedef struct {
    double w_z, z_ref;          /* trunk height */
    double w_o;                 /* orientation error vs upright, yaw 0 */
    double w_v, v_ref;          /* body-frame forward velocity */
    double w_p, goal_xy[2];     /* trunk xy position */
    double w_u;                 /* R = w_u I on (u - u_ref(t)) */
    double w_box, box_goal_xy[2];  /* Q_box || xbar_box - x_box ||_1 (xy) */
    int gait;                   /* 0: u_ref = stand pose; 1: open-loop trot; 2: trot with
                                   Raibert foot-placement feedback */
    double gait_period, gait_hip_amp, gait_knee_amp;
    double stand[3];            /* (abd, hip, knee) stand pose */
    double w_terminal;          /* multiplier of the t = H state terms */
    double raibert_k, raibert_len;  /* gait 2: velocity-error gain (s), effective leg length (m) */
    int z_rel;                  /* 1: z_ref is measured from the ground under the trunk */
} or_cost;

/* ---------------- MPPI parameters ---------------- */
typedef struct {
    int K, H, n_sub, ctrl_steps;  /* samples, horizon (dt steps), sub-steps, control period in dt steps */
    double dt, lambda;
    float sigma[OR_D];
    float q_lo[3], q_hi[3];       /* joint-target clamp per joint type */
    uint64_t seed;
    uint32_t inst;
    int n_prop;                   /* last n_prop samples are drawn around mu_prop */
    int interp;                   /* control representation, OR_INTERP_* */
} or_mppi;

/* Control representations (Sec. III-B; the ablation of Fig. 5): 4 knots at
 * tau_j = j / 3 interpolated by the cubic through them (the default), held
 * (zeroth order: the nearest knot at or before tau) or joined by straight
 * lines; or one target per dt step sampled directly (D = 12 H). */
#define OR_INTERP_CUBIC 0
#define OR_INTERP_ZERO 1
#define OR_INTERP_LINEAR 2
#define OR_INTERP_DIRECT 3

/* spatial algebra */
void or_skew(const real a[3], real S[3][3]);
void or_crm(const real v[6], real M[6][6]);
void or_crf(const real v[6], real M[6][6]);
void or_mcI(real m, const real c[3], const real Ic[3][3], real I[6][6]);
void or_rot_axis(int axis, real th, real E[3][3]);
void or_xform(const real E[3][3], const real r[3], real X[6][6]);
void or_quat_to_R(const real q[4], real R[3][3]);

/* tree */
void or_tree_init(or_tree* t, int floating, double gz);
int  or_tree_add(or_tree* t, int parent, int axis, const double xtree[3], double mass,
                 const double com[3], const double Ic[9]);
int  or_tree_nq(const or_tree* t);
int  or_tree_nv(const or_tree* t);
void or_fk(const or_tree* t, const real* q, real R[][3][3], real p[][3]);
void or_body_vel(const or_tree* t, const real* q, const real* v, real vb[][6]);
void or_aba(const or_tree* t, const real* q, const real* v, const real* tau,
            const real fext[][6], const real* arm, real* acc);
void or_rnea(const or_tree* t, const real* q, const real* v, const real* acc,
             const real fext[][6], const real* arm, real* tau_out);
void or_crba(const or_tree* t, const real* q, const real* arm, real* M);
void or_momentum_world(const or_tree* t, const real* q, const real* v, real h[6]);
void or_momentum_rate_world(const or_tree* t, const real* q, const real* v, const real* acc,
                            real hdot[6]);

/* world */
void or_world_init(or_world* w, const or_params* p);
int  or_world_nx(const or_world* w);
void or_terrain_height(const or_world* w, real x, real y, real* h, real* hx, real* hy);
void or_contact_fext(const or_world* w, const real* x, real fext[][6], real fbox[6]);
void or_substep(const or_world* w, real* x, const real u[OR_NJ], real h);
void or_spline_basis(int H, int t, real B[OR_NKNOT]);
void or_spline_eval(const float* U, real tau, real u[OR_NJ]);
int  or_param_dim(int interp, int H);
void or_interp_basis(int interp, int H, int t, real B[OR_NKNOT]);
void or_controls(int interp, int H, int t, const float* U, real u[OR_NJ]);
void or_gait_ref(const or_cost* c, real t_abs, real uref[OR_NJ]);
void or_gait_ref_x(const or_cost* c, real t_abs, const real* x, real uref[OR_NJ]);
real or_ground_under(const or_world* w, real x, real y);
real or_stage_cost(const or_world* w, const or_cost* c, const real* x, const real* u, real t_abs);
real or_terminal_cost(const or_world* w, const or_cost* c, const real* x);
real or_rollout(const or_world* w, const or_cost* c, int H, int n_sub, real dt, real t0,
                const real* x0, const float* U, real* traj);
real or_rollout_mode(const or_world* w, const or_cost* c, int interp, int H, int n_sub, real dt,
                     real t0, const real* x0, const float* U, real* traj);
void or_rollouts(const or_world* w, const or_cost* c, const or_mppi* m, double t0,
                 const double* x0, int x0_per_sample, const float* U, int n,
                 double* L_out, double* traj, int nthreads);

void or_dt_steps(const or_world* w, const double* X, const double* Ut, long m, int n_sub,
                 double h, double* out, int nthreads);
void or_stage_costs(const or_world* w, const or_cost* c, const double* X, const double* Ut,
                    const double* t_abs, long m, double* out);

/* sampling (FP32 by specification) */
void  or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float or_lnf(float x);
void  or_sincos2pi_u24(uint32_t n24, float* c, float* s);
void  or_box_muller(uint32_t a, uint32_t b, float* e0, float* e1);
void  or_noise(uint64_t seed, uint32_t step, uint32_t inst, uint32_t k, float eps[OR_D]);
void  or_sample(const or_mppi* m, const float* mu, const float* mu_prop,
                uint32_t step, float* U);

/* update (Eq. 1, Eq. 2) and shift */
int  or_update(const float* L, const float* U, int K, double lambda, float mu_out[OR_D],
               double* w_out);
int  or_update_d(const double* L, const float* U, int K, double lambda, float mu_out[OR_D],
                 double* w_out);
void or_shift(const float mu[OR_D], int H, int ctrl_steps, float mu_out[OR_D]);
int  or_update_dim(const double* L, const float* U, int K, int D, double lambda, float* mu_out,
                   double* w_out);
void or_shift_mode(const float* mu, int interp, int H, int ctrl_steps, float* mu_out);
int  or_mppi_step(const or_world* w, const or_cost* c, const or_mppi* m, const double* x0,
                  float* mu, const float* mu_prop, uint32_t step, float u0[OR_NJ],
                  float* L_out, float* U_out, int nthreads);

/* helpers for the Python test harness */
size_t or_world_size(void);
size_t or_tree_size(void);
void or_lnf_many(const float* x, float* y, long n);
void or_sincos_u24_many(const uint32_t* nn, float* c, float* s, long n);
void or_noise_many(uint64_t seed, uint32_t step, uint32_t inst, const uint32_t* ks, long n,
                   float* eps);

#ifdef __cplusplus
}
#endif
#endif
