/*
 * mppi.h -- C ABI of the GB300 (sm_103a) whole-body MPPI hot path.
 *
 * Method: arXiv 2409.10469 (Alvarez-Padilla et al., "Real-Time Whole-Body Control
 * of Legged Robots with Model-Predictive Path Integral Control").
 *   Alg. 1 (Sec. II-B): sample N perturbations of the control mean, simulate each
 *   over T steps, accumulate its cost, weight by Eq. 1, update the mean by Eq. 2,
 *   apply u = mu[0], shift the mean.  Controls are 4 cubic-spline knots of 12 joint
 *   targets (Sec. III-B, Fig. 2) tracked by PD (Sec. IV-A).  Costs: L_walk
 *   (Sec. IV-B) and L_box (Sec. IV-D).  The rollout model replaces MuJoCo
 *   (Sec. III-A): floating-base Featherstone ABA, penalty contacts with regularised
 *   Coulomb friction, semi-implicit Euler with n_sub sub-steps.
 *
 * Conventions shared by every entry point:
 *   - Status codes, never abort/exit; mppi_last_error() gives the text.
 *   - Pointers may be host or device memory: the library asks
 *     cudaPointerGetAttributes and copies host buffers through its own pinned
 *     staging.  The caller owns every pointer it passes; the handle owns its
 *     device workspace.  Calls run on the current device, which must be the
 *     one the handle (batch, network, server) was created on, and device
 *     buffers must be memory of that device or managed memory: another GPU's
 *     memory, or a call made while another device is current, returns
 *     MPPI_ERR_ARG before anything is copied or launched.
 *   - Work is enqueued on the handle's stream (given at creation; NULL = the
 *     legacy default stream).  A call returns once its work is enqueued, except
 *     that results written to HOST memory are complete on return (the call
 *     synchronises the stream).
 *   - A handle is not thread-safe; different handles are independent.
 *   - State x (float): [p(3) world, quat(w,x,y,z) body->world (4), joints(12),
 *     omega body(3), v body(3), joint rates(12)] = 37, plus the free box
 *     [p, quat, omega, v] (13) = 50 when the model has one.  Joint order
 *     FR, FL, RR, RL x (abduction, hip flexion, knee).
 *   - Knots U (float[48]) are [knot j = 0..3][joint 0..11]; knot j sits at
 *     normalised time j/3 of the horizon.
 */
#ifndef MPPI_GB300_H
#define MPPI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mppi_handle_s* mppi_handle;

typedef enum {
    MPPI_OK = 0,
    MPPI_ERR_ARG = 1,        /* invalid argument (null, size out of range, bad layout) */
    MPPI_ERR_OOM = 2,        /* device allocation failed */
    MPPI_ERR_CUDA = 3,       /* a CUDA call failed (text in mppi_last_error) */
    MPPI_ERR_NONFINITE = 4,  /* non-finite state, or every rollout cost non-finite */
    MPPI_ERR_TIMEOUT = 5,    /* a bounded device wait ran out */
    MPPI_ERR_BUSY = 6,       /* admission refused (memory budget) */
    MPPI_ERR_NOTSUP = 7      /* requested feature not available in this library */
} mppi_status;

/* Raw physical description of robot, contacts and terrain.  Derived quantities
 * (spatial inertias) are computed by the library.  The heightfield pointer is
 * read at creation (host or device) and copied into the handle. */
typedef struct {
    double trunk_mass, trunk_size[3];
    double hip_x, hip_y, hip_z;
    double abd_mass, abd_radius;
    double thigh_offset_y;
    double thigh_mass, thigh_length;
    double calf_mass, calf_length;
    double rod_radius;
    double foot_radius;
    int n_trunk_spheres; double trunk_sphere_x[4]; double trunk_sphere_r;
    double gravity;
    double kp, kd, armature;
    double k_contact, c_contact, mu, eps_v;
    int has_box; double box_mass, box_size[3], box_corner_r;
    int terrain;                 /* 0 plane z = 0, 1 heightfield */
    int hf_nx, hf_ny; double hf_cell, hf_x0, hf_y0;
    const float* hf;             /* [hf_ny][hf_nx] heights, row = y */
    int n_static_boxes; double sbox_lo[4][3], sbox_hi[4][3];
} mppi_model_t;

/* L_walk (Sec. IV-B) + L_box (Sec. IV-D) weights and references.  gait 2 is the
 * trot reference with the Raibert heuristic's foot placement (Sec. IV-B): a
 * swinging leg's hip-flexion target moves by -dx / raibert_len (clamped to
 * 0.4 rad, weighted by the swing profile), dx = (gait_period / 4) v_x +
 * raibert_k (v_x - v_ref), v_x the trunk's body-frame forward velocity.  z_rel:
 * the height reference counts from the ground under the trunk (terrain or the
 * top of a static box containing the trunk's xy), for climbing (Sec. IV-C). */
typedef struct {
    double w_z, z_ref, w_o, w_v, v_ref, w_p, goal_xy[2], w_u, w_box, box_goal_xy[2];
    int gait;                    /* 0 stand reference, 1 open-loop trot, 2 trot + Raibert feedback */
    double gait_period, gait_hip_amp, gait_knee_amp;
    double stand[3];
    double w_terminal;
    double raibert_k, raibert_len;
    int z_rel;
} mppi_cost_t;

/* Control representation of a sample (Sec. III-B, the ablation of Fig. 5).
 * The knot representations sample 4 knots x 12 joints at normalised times
 * tau_j = j / 3 (tau_t = t / (H - 1) for dt step t) and interpolate them:
 *   CUBIC  the cubic through the 4 knots (Lagrange basis; the paper's choice);
 *   ZERO   zeroth-order hold: knot j = floor(3 t / (H - 1)) (integer division);
 *   LINEAR straight lines between knots j and j + 1 (j <= 2) at that t.
 * DIRECT samples one 12-joint target per dt step: D = 12 H parameters, joint i
 * perturbed with sigma[i] (the first knot's).  D = 48 for the knot forms. */
#define MPPI_INTERP_CUBIC 0
#define MPPI_INTERP_ZERO 1
#define MPPI_INTERP_LINEAR 2
#define MPPI_INTERP_DIRECT 3

/* Alg. 1 inputs N (= K), T (= H), lambda, Sigma (diagonal sigma), plus the model's
 * sub-step count and the control period in dt steps. */
typedef struct {
    int K, H, n_sub, ctrl_steps;
    double dt, lambda;
    float sigma[48];
    float q_lo[3], q_hi[3];      /* knot clamp per joint type */
    uint64_t seed;               /* Philox4x32-10 key */
    uint32_t inst;               /* instance id (Philox counter word 3) */
    int n_prop;                  /* last n_prop samples centre on a proposal mean */
    int block;                   /* rollout kernel block size in threads (0 = default) */
    int interp;                  /* MPPI_INTERP_* (0 = cubic) */
} mppi_config_t;

/* Create a controller: copies model, cost and config, derives the model's
 * device constants, allocates its workspace (U[K][D], L[K], mu[D], u0, status;
 * D = mppi_param_dim) for up to cfg->K samples.  stream: a cudaStream_t or NULL.
 * Errors: ARG (K < 1, H < 2, n_sub < 1, dt <= 0, lambda <= 0, bad terrain,
 * unknown interp, n_prop > 0 with DIRECT), OOM, CUDA. */
mppi_status mppi_create(const mppi_model_t* model, const mppi_cost_t* cost,
                        const mppi_config_t* cfg, void* stream, mppi_handle* out);

/* Free the handle and its device memory (synchronises its stream). */
mppi_status mppi_destroy(mppi_handle h);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char* mppi_last_error(mppi_handle h);

/* Parameters per sample D: 48 (4 knots x 12 joints) for the knot representations,
 * 12 H for DIRECT.  Every float[48] / float[n][48] below is float[D] / float[n][D]
 * for a DIRECT handle (u0 stays float[12]). */
int mppi_param_dim(mppi_handle h);

/* Nominal knots mu (float[48], host or device): write / read. */
mppi_status mppi_set_nominal(mppi_handle h, const float* mu);
mppi_status mppi_get_nominal(mppi_handle h, float* mu_out);
/* The samples of the handle's last control step (mppi_step, mppi_step_proposal,
 * or a batch step the handle took part in): the K perturbed parameter vectors
 * and their rollout costs -- the inputs of Eq. 1 / Eq. 2 (Alg. 1's sampled
 * controls and their total costs).  U_out (float[K][D]) and L_out (float[K]),
 * host or device, either may be NULL; the handle's workspace is copied on its
 * stream, and the call returns once host outputs are written.  Undefined before
 * the first step (the workspace is not cleared). */
mppi_status mppi_get_samples(mppi_handle h, float* U_out, float* L_out);

/* Alg. 1 sampling step (Sec. II-B; noise generator per the model spec):
 * U[k] = clamp(mu + sigma * eps_k), eps_k = Box-Muller(Philox4x32-10(key = seed,
 * counter = (g, k, step, inst))), sample 0 = mu; with mu_prop != NULL the last
 * n_prop samples centre on mu_prop (the first of them is mu_prop itself).
 * U_out: float[K][48] (host or device), or NULL to fill the handle's own buffer. */
mppi_status mppi_sample(mppi_handle h, uint32_t step, const float* mu_prop, float* U_out);

/* Alg. 1 simulate-and-cost step: roll out n knot vectors U (float[n][48]; NULL =
 * the handle's sampled buffer, n <= K) from x0 (float[nx], or float[n][nx] when
 * x0_per_sample) over H dt steps of n_sub sub-steps, starting at absolute time t0
 * (phase of the gait reference).  L_out: float[n] costs (L_walk + L_box, NULL =
 * the handle's buffer).  traj_out: optional float[n][H + 1][nx] states x_0..x_H.
 * Errors: ARG, NONFINITE (x0 not finite), CUDA. */
mppi_status mppi_rollouts(mppi_handle h, const float* x0, int x0_per_sample, const float* U,
                          int n, double t0, float* L_out, float* traj_out);

/* Eq. 1 + Eq. 2 + apply + shift: weights exp(-(L - L_min)/lambda) over finite
 * costs (exponent and exp in FP64, the sums in compensated float-float pairs),
 * mu' = sum w U / sum w, u0 = mu'[knot 0] (the first target for DIRECT),
 * then the nominal becomes shifted(mu').  L (float[n]) and U (float[n][48]) may be
 * NULL for the handle's own buffers.  mu_out (float[48], the updated mean before
 * the shift), u0_out (float[12]) optional.  Returns NONFINITE and keeps mu when
 * no cost is finite. */
mppi_status mppi_update(mppi_handle h, const float* L, const float* U, int n, float* mu_out,
                        float* u0_out);

/* One full control step of Alg. 1 at control index `step` (gait time
 * step * ctrl_steps * dt): sample, roll out from x0 (float[nx]), update, shift.
 * u0_out: float[12] joint targets to apply; mu_out optional float[48] (updated
 * mean before the shift).  With host outputs the call returns after the step
 * completed.  One kernel for the knot representations: the rollout kernel draws
 * the knots itself (bit-identical to mppi_sample, left in the handle's U) and
 * ends with the update (each CTA sums its rollouts' weights around its own cost
 * minimum in FP64, the last CTA combines them); three kernels for direct
 * targets. */
mppi_status mppi_step(mppi_handle h, const float* x0, uint32_t step, float* u0_out,
                      float* mu_out);

/* Per-kernel device time of the last mppi_step, measured with CUDA events on
 * the handle's stream when timing is on: ms[0] sample, ms[1] rollout, ms[2]
 * update (for the knot forms sampling and update run inside the rollout kernel,
 * so ms[0] and ms[2] are 0).  Timing is off by default (events add a few
 * microseconds). */
mppi_status mppi_set_timing(mppi_handle h, int on);
mppi_status mppi_get_timings(mppi_handle h, float ms[3]);

/* Number of kernels the library launched on this handle since creation. */
mppi_status mppi_launch_count(mppi_handle h, uint64_t* count);

/* State size of the handle's model: 37, or 50 with the free box. */
int mppi_state_size(mppi_handle h);

/* ------------------------------------------------------------------ batches
 * Many controllers (handles of any K, H, terrain, task) stepped together: one
 * persistent kernel per control step runs Alg. 1 for every active instance
 * (sampling in-kernel with the same bit-exact noise, the same rollout
 * arithmetic as mppi_rollouts, and each instance's Eq. 1/Eq. 2 update + shift
 * in a fixed order by the block that finishes its last rollouts), captured in a
 * CUDA graph.  An instance's result does not depend on the other instances in
 * the batch.  The handles must outlive the batch; their nominals are updated in
 * place exactly as mppi_step would. */
typedef struct mppi_batch_s* mppi_batch;

/* Batch of n handles (all on the current device).  stream: cudaStream_t or NULL. */
mppi_status mppi_batch_create(const mppi_handle* hs, int n, void* stream, mppi_batch* out);
mppi_status mppi_batch_destroy(mppi_batch b);
const char* mppi_batch_last_error(mppi_batch b);

/* One control step of every active instance.  active: host int[n] (non-zero =
 * step this instance; NULL = all); x0s: float[n][50] host or device (row i uses
 * its first nx_i entries); steps: host uint32[n] control-step index of each
 * instance (its Philox counter word 2 and gait time), NULL = unchanged;
 * u0s: optional float[n][12] host or device (rows of inactive instances keep
 * their last value, zero before an instance's first step).  Host outputs are
 * complete on return. */
mppi_status mppi_batch_step(mppi_batch b, const int* active, const float* x0s, const uint32_t* steps,
                            float* u0s);

/* Block shape of the persistent kernel: block in {64, 128, 256} threads (block/4
 * rollouts per work item), blocks_per_sm up to the occupancy limit. */
mppi_status mppi_batch_set_shape(mppi_batch b, int block, int blocks_per_sm);
mppi_status mppi_batch_get_shape(mppi_batch b, int* block, int* blocks_per_sm);

/* Autotuner: times every candidate shape (trials steps each, CUDA events, from
 * the same nominals, which are restored afterwards) on this batch from x0s and
 * keeps the fastest.  Outputs (optional): the chosen shape and its step time. */
mppi_status mppi_batch_autotune(mppi_batch b, const float* x0s, int trials, int* block_out,
                                int* bpsm_out, float* best_ms_out);

/* After a step: every instance's updated mean before the shift (mu_upds,
 * float[n][48]) and its shifted nominal (nominals, float[n][48]); host or
 * device, either may be NULL. */
mppi_status mppi_batch_get_means(mppi_batch b, float* mu_upds, float* nominals);

/* Number of graph launches (one per mppi_batch_step). */
mppi_status mppi_batch_launch_count(mppi_batch b, uint64_t* count);

/* *shared = 1 when every instance of the batch simulates the same model (equal
 * values, heights and static boxes, whichever handle holds them) under the
 * same cost: the persistent kernel then takes both from its launch parameters
 * (the path the single-instance kernel uses) instead of each work item's copy
 * in shared memory.  Results are bit-identical either way. */
mppi_status mppi_batch_shared_model(mppi_batch b, int* shared);

/* ------------------------------------------------------------------ serving
 * Continuous batching of control-step requests from many robots.  A robot is a
 * controller handle (its nominal stays on the device between requests).  The
 * server admits queued requests in arrival order while their workspace (K x 49
 * floats per solve) fits a device pool of budget_bytes, launches the admitted
 * set as one persistent multi-instance step on one of two streams (so requests
 * admitted while another launch runs overlap with it on the GPU), and retires
 * launches when their completion event fires.  A robot's control is the same
 * alone and in any mix.  All calls are host-side and non-blocking except
 * drain; tick must be called to make progress (it never waits on the GPU). */
typedef struct mppi_server_s* mppi_server;

typedef struct {
    uint64_t submitted, completed, launches, busy_rejects, queued, in_flight;
    uint64_t pool_bytes, pool_in_use, pool_peak;
    double rollout_steps;                          /* sum of K * H over completed requests */
    double latency_p50, latency_p99, latency_max;  /* seconds, submit -> observed completion */
} mppi_server_stats_t;

/* budget_bytes: device pool for solve workspace; max_robots; max_samples: the
 * largest K of any robot.  Errors: ARG, OOM. */
mppi_status mppi_server_create(size_t budget_bytes, int max_robots, int max_samples, mppi_server* out);
mppi_status mppi_server_destroy(mppi_server s);
const char* mppi_server_last_error(mppi_server s);
/* Register a robot (its handle must outlive the server).  ARG if one of its
 * solves alone exceeds the budget, or if the handle was created on another
 * device than the server. */
mppi_status mppi_server_add_robot(mppi_server s, mppi_handle h, int* robot_id);
/* Queue one control step of `robot` from host state x0 (float[nx]) at control
 * index `step`.  BUSY if the robot already has a request queued or in flight;
 * NONFINITE if x0 is not finite; ARG if x0 is device memory. */
mppi_status mppi_server_submit(mppi_server s, int robot, const float* x0, uint32_t step);
/* Retire finished launches, admit and launch queued requests. */
mppi_status mppi_server_tick(mppi_server s, int* completed);
/* ready = 1 and the control (float[12], host memory) and submit-to-completion
 * latency when a new result is waiting; ready = 0 otherwise. */
mppi_status mppi_server_poll(mppi_server s, int robot, float* u0_out, double* latency_s, int* ready);
mppi_status mppi_server_stats(mppi_server s, mppi_server_stats_t* out);
mppi_status mppi_server_reset_stats(mppi_server s);
/* Block until every queued and in-flight request has completed. */
mppi_status mppi_server_drain(mppi_server s);

/* ------------------------------------------------------------------ proposal network
 * The learned sampling distribution that the paper leaves to future work
 * (Sec. V-B; offline-learned distributions are cited in Sec. II-B): an MLP
 * 62 -> 256 -> 256 -> 256 -> 48 with GELU (x Phi(x)), BF16 weights and activations,
 * FP32 accumulation, trained and run on the tcgen05 tensor cores.  Parameters
 * are one flat FP32 array: W1 [256][62], b1 [256], W2 [256][256], b2, W3 [256][256],
 * b3, W4 [48][256], b4 [48] (row = output unit); the network keeps FP32 master
 * copies and refreshes BF16 copies for its GEMMs. */
typedef struct mppi_mlp_s* mppi_mlp;

mppi_status mppi_mlp_create(int max_batch, mppi_mlp* out);
mppi_status mppi_mlp_destroy(mppi_mlp net);
const char* mppi_mlp_last_error(mppi_mlp net);
long mppi_mlp_param_count(mppi_mlp net);
/* params: float[param_count], host or device; resets the optimiser state. */
mppi_status mppi_mlp_set_params(mppi_mlp net, const float* params, void* stream);
mppi_status mppi_mlp_get_params(mppi_mlp net, float* params, void* stream);
/* Y[B][48] = MLP(X[B][62]) (host or device buffers; B <= max_batch). */
mppi_status mppi_mlp_forward(mppi_mlp net, const float* X, int B, float* Y, void* stream);
/* One training step on (X[B][62], T[B][48]): mean-squared-error loss, backward
 * pass on the tensor cores, AdamW (beta 0.9 / 0.999, eps 1e-8) when lr > 0.
 * loss_out (float), grad_out (float[param_count], the gradient before the
 * update) optional.  TIMEOUT if a tensor-core wait ran out. */
mppi_status mppi_mlp_train_step(mppi_mlp net, const float* X, const float* T, int B, float lr,
                                float weight_decay, float* loss_out, float* grad_out, void* stream);
/* Failure-detection self-test: runs both tensor-core GEMM kernels (the
 * thread-staged one and the TMA-fed pipeline) with their completion signals
 * withheld, so their bounded waits run out; each kernel records the timeout,
 * lets its copies in flight land, releases its tensor memory and returns.  Then
 * the small-batch cluster forward with its first layer's weight copy withheld:
 * its waits run out, it records that and returns in step with its cluster.
 * Expected result: MPPI_ERR_TIMEOUT (all three timed out), with the CUDA
 * context still usable afterwards. */
mppi_status mppi_selftest_wait_timeout(void* stream);

/* Noise self-test (the sampler's Box-Muller transform, Sec. II-B sampling step,
 * over its whole input domain): for every 24-bit i, radius[i] = sqrt(-2 ln u1)
 * with u1 = (i + 1) 2^-24, and cosv[i], sinv[i] = cos, sin of 2 pi i 2^-24,
 * computed by the device code the sampling kernels use.  radius, cosv, sinv:
 * device float[2^24] each (caller-owned).  ARG for null or host pointers;
 * asynchronous on `stream`. */
mppi_status mppi_selftest_noise_tables(float* radius, float* cosv, float* sinv, void* stream);

/* The network's input for n states X (float[n][nx], host or device) of this
 * handle's robot and task at control index `step`: F (float[n][62], host or
 * device) = trunk height, attitude (w >= 0), joints, velocities, joint rates
 * x 0.1, box pose/velocity relative to the trunk, box-goal and trunk-goal
 * offsets, gait phase (sin, cos), gravity in the trunk frame, box heading,
 * the two xy distances and a constant 1. */
mppi_status mppi_features(mppi_handle h, const float* X, int n, uint32_t step, float* F);
/* Proposal mean for the handle's next steps (float[48], host or device; NULL
 * stops using it): mppi_step and batches then draw the last n_prop samples
 * around it (the first of them is the proposal itself); a non-finite entry
 * falls back to the plain mean.  ARG if the handle has n_prop = 0. */
mppi_status mppi_set_proposal(mppi_handle h, const float* mu_prop);
/* ---- K-sharded control step (one controller over several GPUs or processes).
 * Alg. 1's K samples are independent until Eq. 1, whose weights factor as
 * exp(-(L_k - L_min) / lambda) = exp(-(L_k - m_r) / lambda) exp(-(m_r - L_min) / lambda)
 * for any shard minimum m_r, so a step can be split by sample range: every rank
 * holds a handle with the same configuration, seed and nominal, calls
 * mppi_step_partial on its own range [k0, k0 + n) of the K samples (the same
 * Philox stream: sample k is the same knot vector whichever rank draws it),
 * takes L_min = min over ranks of part[0] (an all-reduce(min)), scales its
 * part[1 .. 49] by exp(-(part[0] - L_min) / lambda) (0 when part[0] is not
 * finite), sums them over ranks (an all-reduce(sum) of 49 doubles) and calls
 * mppi_step_finalize with the sums: every rank then holds the same mu', u0 and
 * shifted nominal -- those of mppi_step on all K samples, up to the order of
 * the sums.  Knot representations only (ARG for DIRECT).
 * mppi_step_partial: x0 float[nx] host or device; the step's samples k0 ..
 * k0 + n - 1 (0 <= k0, 1 <= n, k0 + n <= K) are drawn, rolled out and weighted
 * around their own finite-cost minimum m; part_out double[MPPI_SHARD_PARTIAL]
 * (host or device) receives (m, Z = sum_k w_k, S[48] = sum_k w_k U_k), m = +inf
 * and Z = S = 0 when no cost of the range is finite.  Host outputs are written
 * on return.  The handle's nominal is not changed.
 * mppi_step_finalize: sums double[49] (Z, S[48]) host or device, combined over
 * every rank relative to the global L_min: mu' = S / Z, the applied u0, the
 * shifted nominal (kept and NONFINITE when Z is not positive and finite);
 * u0_out / mu_out as in mppi_step. */
#define MPPI_SHARD_PARTIAL 50
mppi_status mppi_step_partial(mppi_handle h, const float* x0, uint32_t step, int k0, int n, double* part_out);
mppi_status mppi_step_finalize(mppi_handle h, const double* sums, float* u0_out, float* mu_out);

/* The learned-proposal form's control step in one call: the features of x0
 * (float[nx], host or device) at control index `step`, the network's forward on
 * them (one small-batch kernel computes both), the result taken as the proposal
 * mean, and mppi_step -- all enqueued on the handle's stream, with no host round
 * trip in between (host outputs synchronise as in mppi_step).  Equal to mppi_features ->
 * mppi_mlp_forward -> mppi_set_proposal -> mppi_step on the same inputs.  The
 * network's parameters must be complete (mppi_mlp_set_params synchronises; a
 * training step still running on another stream races with this call).  ARG if
 * the handle has n_prop = 0 or uses direct targets; NONFINITE as mppi_step. */
mppi_status mppi_step_proposal(mppi_handle h, mppi_mlp net, const float* x0, uint32_t step, float* u0_out,
                               float* mu_out);
/* D[M][N] = A[M][K] B[N][K]^T with BF16 inputs (raw uint16 bits) and FP32
 * accumulation on the tcgen05 tensor cores -- the network's GEMM; device
 * buffers, N <= 256, row-major with K contiguous.  K a multiple of 8, N a
 * multiple of 4 and 16-byte aligned buffers take the TMA-fed pipelined kernel,
 * other shapes the thread-staged one.  Synchronous: returns once D is written
 * (TIMEOUT if a tensor-core wait ran out). */
mppi_status mppi_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                              void* stream);

/* The update of mppi_update (Eq. 1 + Eq. 2 + apply + shift) without a handle and
 * without allocating anything.  The paper has no counterpart: this is for
 * callers that must not allocate device memory when they run -- a hard
 * real-time control loop that may not block in the driver's allocator, code
 * running inside another framework's memory pool, or a runtime that forbids
 * cudaMalloc after start-up.  They pass every buffer; the call's scratch (a row
 * of 50 doubles of partial sums for each of at most 128 CTAs, and a completion
 * counter) is a fixed 51,456-byte device array compiled into the library,
 * which every GPU that loads the library keeps until the process exits.  n only
 * sets how many samples each CTA sums, so every n up to MPPI_NOALLOC_MAX_N fits.
 *   L (float[n]), U (float[n][48], 16-byte aligned): costs and knots, device.
 *   interp: the knot representation the knots belong to (MPPI_INTERP_CUBIC,
 *   _ZERO or _LINEAR): the shift re-samples that representation's interpolant.
 *   mu_in (float[48]): the current nominal (kept if every cost is non-finite).
 *   mu_out (float[48]): the shifted nominal; may equal mu_in.
 *   mu_upd_out (float[48], optional): the updated mean before the shift.
 *   u0_out (float[12]): the control to apply; status_out (int, optional): 0, or
 *   4 when every cost is non-finite.  All pointers are device memory of the
 *   current device (or managed memory).
 *   stream: a cudaStream_t or NULL; the call only enqueues work.
 * The first call on a device looks up the array's device address with that
 * device current, so make it before any stream capture.  Calls share the one
 * array, whose completion counter each call clears before its kernel: calls
 * that overlap on the GPU (different streams, or threads without ordering) race
 * and corrupt each other's results.
 * Errors: MPPI_ERR_ARG when n < 1 or n > MPPI_NOALLOC_MAX_N, H < 2,
 * ctrl_steps < 1, lambda <= 0, interp is not a knot representation, a buffer is
 * not device memory of the current device or U is misaligned; MPPI_ERR_CUDA
 * when a CUDA call fails.  No cudaMalloc, cudaFree or other allocating call is
 * made. */
#define MPPI_NOALLOC_MAX_N (1 << 20)
mppi_status mppi_update_noalloc(const float* L, const float* U, int n, int H, int ctrl_steps,
                                double lambda, int interp, const float* mu_in, float* mu_out,
                                float* mu_upd_out, float* u0_out, int* status_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
