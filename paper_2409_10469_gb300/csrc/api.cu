// api.cu -- C ABI (include/mppi.h) of the sm_103a MPPI hot path.
//
// Owns the controller handle: derived FP32 model constants (spatial inertias
// built here from the raw description), device workspace, the caller's stream,
// host<->device marshalling of host pointers, and per-kernel event timing.
// Every step of the path runs in the kernels of sample.cu, rollout.cu and
// update.cu; nothing here computes on the host beyond argument preparation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <string>
#include <cstddef>
#include <vector>

#include "handle.h"
#include "memkind.h"

using namespace mppi;

// ------------------------------------------------------------------ helpers

static mppi_status fail(mppi_handle h, mppi_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

static mppi_status cuda_fail(mppi_handle h, cudaError_t e, const char* where) {
    return fail(h, MPPI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);    \
    } while (0)

// true when p is memory of the current device (or managed memory); host memory
// (pageable or pinned) -> false.  Another GPU's memory never reaches here: every
// entry point rejects it first (local_call).
static bool is_device(const void* p) { return is_local(p); }

// The checks every call taking buffers makes before its first copy or launch:
// the handle's device is the current one (its workspace lives there), and no
// buffer is device memory of another GPU.
static mppi_status local_call(mppi_handle h, std::initializer_list<const void*> bufs) {
    const int dev = current_device();
    if (dev < 0) return fail(h, MPPI_ERR_CUDA, "cudaGetDevice failed");
    if (dev != h->device) return fail(h, MPPI_ERR_ARG, "the handle's device is not the current device");
    if (any_foreign(dev, bufs)) return fail(h, MPPI_ERR_ARG, "a buffer is memory of another GPU");
    return MPPI_OK;
}
#define LOCAL_CALL(...)                                              \
    do {                                                             \
        const mppi_status s_ = local_call(h, {__VA_ARGS__});         \
        if (s_ != MPPI_OK) return s_;                                \
    } while (0)

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// inertia of a body with its centre of mass on the frame's z axis at cz and a
// diagonal rotational inertia Icd there, about the frame origin
static BodyI body_inertia(double m, double cz, const double Icd[3]) {
    BodyI I;
    I.ax = (float)(Icd[0] + m * cz * cz);
    I.ay = (float)(Icd[1] + m * cz * cz);
    I.az = (float)Icd[2];
    I.m = (float)m;
    I.mcz = (float)(m * cz);
    return I;
}

// implicit-PD armature of one sub-step: h (kd + h kp) + a0
double mppi_armature(const mppi_model_t& p, double h) { return h * (p.kd + h * p.kp) + p.armature; }
static double armature(const mppi_model_t& p, double h) { return mppi_armature(p, h); }

static void derive_model(const mppi_model_t& p, double h, DevModel& d) {
    memset(&d, 0, sizeof(d));
    const double a = p.trunk_size[0], b = p.trunk_size[1], c = p.trunk_size[2], m = p.trunk_mass;
    d.tr_Ic[0] = (float)(m * (b * b + c * c) / 12.0);
    d.tr_Ic[1] = (float)(m * (a * a + c * c) / 12.0);
    d.tr_Ic[2] = (float)(m * (a * a + b * b) / 12.0);
    d.tr_m = (float)m;
    const double ih = 0.4 * p.abd_mass * p.abd_radius * p.abd_radius;
    const double Ihip[3] = {ih, ih, ih};
    d.I_hip = body_inertia(p.abd_mass, 0.0, Ihip);
    const double tl = p.thigh_length, cl = p.calf_length, rr = p.rod_radius;
    const double It[3] = {p.thigh_mass * tl * tl / 12.0, p.thigh_mass * tl * tl / 12.0, p.thigh_mass * rr * rr / 2.0};
    d.I_thigh = body_inertia(p.thigh_mass, -0.5 * tl, It);
    const double Ic[3] = {p.calf_mass * cl * cl / 12.0, p.calf_mass * cl * cl / 12.0, p.calf_mass * rr * rr / 2.0};
    d.I_calf = body_inertia(p.calf_mass, -0.5 * cl, Ic);
    {
        // the calf has no children: its articulated inertia is its rigid inertia
        // and its projection I - U U^T / D (U = I e_y, D = U_y + armature) is a
        // constant of the model and the sub-step
        const double mc = p.calf_mass, cz = -0.5 * cl;
        const double ax = Ic[0] + mc * cz * cz, ay = Ic[1] + mc * cz * cz, az = Ic[2], mcz = mc * cz;
        double A[3][3] = {{ax, 0, 0}, {0, ay, 0}, {0, 0, az}};
        double B[3][3] = {{0, -mcz, 0}, {mcz, 0, 0}, {0, 0, 0}};
        double C[3][3] = {{mc, 0, 0}, {0, mc, 0}, {0, 0, mc}};
        const double U[6] = {A[0][1], A[1][1], A[2][1], B[1][0], B[1][1], B[1][2]};
        const double D = U[1] + armature(p, h);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                A[i][j] -= U[i] * U[j] / D;
                B[i][j] -= U[i] * U[3 + j] / D;
                C[i][j] -= U[3 + i] * U[3 + j] / D;
            }
        for (int i = 0; i < 3; i++)
            for (int j = i; j < 3; j++) {
                d.Ia_calf.A[sidx(i, j)] = (float)A[i][j];
                d.Ia_calf.C[sidx(i, j)] = (float)C[i][j];
            }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) d.Ia_calf.B[i][j] = (float)B[i][j];
        d.calf_D_inv = (float)(1.0 / D);
    }
    // legs FR, FL, RR, RL: front +x / rear -x, right -y / left +y (signs in the kernel)
    d.hip_x = (float)p.hip_x;
    d.hip_y = (float)p.hip_y;
    d.hip_z = (float)p.hip_z;
    d.thigh_y = (float)p.thigh_offset_y;
    d.r_knee[0] = 0.f; d.r_knee[1] = 0.f; d.r_knee[2] = (float)(-tl);
    d.foot[0] = 0.f; d.foot[1] = 0.f; d.foot[2] = (float)(-cl);
    d.foot_r = (float)p.foot_radius;
    d.n_tsph = p.n_trunk_spheres;
    for (int s = 0; s < 4; s++) d.tsph_x[s] = s < p.n_trunk_spheres ? (float)p.trunk_sphere_x[s] : 0.f;
    d.tsph_r = (float)p.trunk_sphere_r;
    d.gz = (float)(-p.gravity);
    d.kp = (float)p.kp; d.kd = (float)p.kd; d.arm0 = (float)p.armature;
    d.kc = (float)p.k_contact; d.cc = (float)p.c_contact; d.mu = (float)p.mu;
    d.eps2 = (float)(p.eps_v * p.eps_v);
    d.terrain = p.terrain;
    d.hf_nx = p.hf_nx; d.hf_ny = p.hf_ny;
    d.hf_cell = (float)p.hf_cell;
    d.hf_inv_cell = p.hf_cell > 0 ? (float)(1.0 / p.hf_cell) : 0.f;
    d.hf_x0 = (float)p.hf_x0; d.hf_y0 = (float)p.hf_y0;
    d.n_sbox = p.n_static_boxes;  // the boxes themselves are filled in by mppi_create
    d.has_box = p.has_box;
    if (p.has_box) {
        d.box_m = (float)p.box_mass;
        d.box_inv_m = (float)(1.0 / p.box_mass);
        const double X = p.box_size[0], Y = p.box_size[1], Z = p.box_size[2];
        const double I3[3] = {p.box_mass * (Y * Y + Z * Z) / 12.0, p.box_mass * (X * X + Z * Z) / 12.0,
                              p.box_mass * (X * X + Y * Y) / 12.0};
        for (int k = 0; k < 3; k++) {
            d.box_half[k] = (float)(0.5 * p.box_size[k]);
            d.box_Ic[k] = (float)I3[k];
            d.box_inv_Ic[k] = (float)(1.0 / I3[k]);
        }
        d.box_cr = (float)p.box_corner_r;
    }
    d.nx = p.has_box ? NX_BOX : NX_ROBOT;
}

static void derive_cost(const mppi_cost_t& c, DevCost& d) {
    d.w_z = (float)c.w_z; d.z_ref = (float)c.z_ref; d.w_o = (float)c.w_o;
    d.w_v = (float)c.w_v; d.v_ref = (float)c.v_ref; d.w_p = (float)c.w_p;
    d.goal_x = (float)c.goal_xy[0]; d.goal_y = (float)c.goal_xy[1];
    d.w_u = (float)c.w_u; d.w_box = (float)c.w_box;
    d.box_gx = (float)c.box_goal_xy[0]; d.box_gy = (float)c.box_goal_xy[1];
    d.gait = c.gait;
    d.two_pi_over_period = c.gait_period > 0 ? (float)(2.0 * M_PI / c.gait_period) : 0.f;
    d.hip_amp = (float)c.gait_hip_amp; d.knee_amp = (float)c.gait_knee_amp;
    for (int i = 0; i < 3; i++) d.stand[i] = (float)c.stand[i];
    d.w_term = (float)c.w_terminal;
    d.quarter_period = (float)(0.25 * c.gait_period);
    d.raibert_k = (float)c.raibert_k;
    d.inv_raibert_len = c.raibert_len > 0 ? (float)(1.0 / c.raibert_len) : 0.f;
    d.z_rel = c.z_rel;
}

// gait time of step 0 of a horizon starting at absolute time t0, reduced
// modulo the gait period so that FP32 keeps its resolution over long runs
float mppi_reduce_t0(const mppi_handle h, double t0) {
    const double P = h->cost_in.gait_period;
    if ((h->cost_in.gait == 1 || h->cost_in.gait == 2) && P > 0) return (float)fmod(t0, P);
    return (float)t0;
}

// a float input of n values: device pointer as is, host data copied to dst
static mppi_status stage_in(mppi_handle h, const float* src, size_t n, float* dst, const float** out) {
    if (is_device(src)) {
        *out = src;
        return MPPI_OK;
    }
    CK(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    *out = dst;
    return MPPI_OK;
}

static bool all_finite(const float* p, size_t n) {
    for (size_t i = 0; i < n; i++)
        if (!isfinite(p[i])) return false;
    return true;
}

// Knot weights of every dt step t of an H-step horizon for a knot representation
// (Sec. III-B; Fig. 5's forms), in double, rounded once: knots at tau_j = j / 3,
// tau_t = t / (H - 1).  Cubic: the Lagrange basis of the 4 knots.  Zeroth order:
// knot j = floor(3 t / (H - 1)) (integer division; 3 at the end).  Linear: knots
// j and j + 1 (j <= 2) with weights 1 - f and f, f = (3 t - j (H - 1)) / (H - 1).
static void knot_weights(int interp, int H, std::vector<float>& B) {
    B.assign((size_t)4 * H, 0.f);
    if (interp == MPPI_INTERP_DIRECT) return;
    for (int t = 0; t < H; t++) {
        double w[4] = {0, 0, 0, 0};
        if (interp == MPPI_INTERP_CUBIC) {
            const double tau = H > 1 ? (double)t / (double)(H - 1) : 0.0;
            for (int j = 0; j < 4; j++) {
                double b = 1.0;
                for (int m = 0; m < 4; m++)
                    if (m != j) b *= (tau - m / 3.0) / (j / 3.0 - m / 3.0);
                w[j] = b;
            }
        } else {
            const int den = H > 1 ? H - 1 : 1;
            int j = (3 * t) / den;
            if (interp == MPPI_INTERP_ZERO) {
                w[j > 3 ? 3 : j] = 1.0;
            } else {
                if (j > 2) j = 2;
                const double f = (double)(3 * t - j * den) / (double)den;
                w[j] = 1.0 - f;
                w[j + 1] = f;
            }
        }
        for (int j = 0; j < 4; j++) B[(size_t)4 * t + j] = (float)w[j];
    }
}

static_assert(MPPI_INTERP_CUBIC == INTERP_CUBIC && MPPI_INTERP_ZERO == INTERP_ZERO &&
                  MPPI_INTERP_LINEAR == INTERP_LINEAR && MPPI_INTERP_DIRECT == INTERP_DIRECT,
              "representation codes of the ABI and the kernels agree");

// ------------------------------------------------------------------ ABI

// threads per block of the rollout kernel (4 per rollout)
static int rollout_block_cfg(const mppi_config_t& c) { return c.block ? c.block : 128; }
// scratch of the update fused into the control step's rollout launch (0 when the
// grid is too large to fuse)
static size_t fused_part_doubles(const mppi_config_t& c) {
    const int g = rollout_grid(c.K, rollout_block_cfg(c));
    return g <= FUSE_MAX_CTAS ? (size_t)g * FUSE_W : 0;
}

// FNV-1a (64-bit) over the model's values -- the pointer fields (device copies of
// the heights and boxes, which every handle owns) are left out by offset ranges,
// so no struct padding enters the hash -- then over the heights and boxes
// themselves.  Handles with equal keys simulate the same model.
static uint64_t fnv1a(uint64_t k, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
        k ^= c[i];
        k *= 1099511628211ull;
    }
    return k;
}
static uint64_t model_key(const DevModel& m, const std::vector<float>& heights, const float* boxes, size_t nbox) {
    const char* b = reinterpret_cast<const char*>(&m);
    uint64_t k = 1469598103934665603ull;
    k = fnv1a(k, b, offsetof(DevModel, hf_y0) + sizeof(float));
    k = fnv1a(k, b + offsetof(DevModel, n_sbox), sizeof(int));
    k = fnv1a(k, b + offsetof(DevModel, has_box), offsetof(DevModel, nx) + sizeof(int) - offsetof(DevModel, has_box));
    k = fnv1a(k, heights.data(), heights.size() * sizeof(float));
    return fnv1a(k, boxes, nbox * sizeof(float));
}

extern "C" mppi_status mppi_create(const mppi_model_t* model, const mppi_cost_t* cost, const mppi_config_t* cfg,
                                   void* stream, mppi_handle* out) {
    if (!model || !cost || !cfg || !out) return MPPI_ERR_ARG;
    *out = nullptr;
    if (cfg->K < 1 || cfg->H < 2 || cfg->n_sub < 1 || !(cfg->dt > 0) || !(cfg->lambda > 0) ||
        cfg->ctrl_steps < 1 || cfg->n_prop < 0 || cfg->n_prop >= cfg->K || cfg->K > (1 << 24))
        return MPPI_ERR_ARG;
    if (cfg->block != 0 && (cfg->block % 32 != 0 || cfg->block < 32 || cfg->block > 256)) return MPPI_ERR_ARG;
    if (cfg->interp < MPPI_INTERP_CUBIC || cfg->interp > MPPI_INTERP_DIRECT) return MPPI_ERR_ARG;
    if (cfg->interp == MPPI_INTERP_DIRECT && (cfg->n_prop > 0 || cfg->H > (1 << 16))) return MPPI_ERR_ARG;
    if (model->terrain == 1 && (!model->hf || model->hf_nx < 2 || model->hf_ny < 2 || !(model->hf_cell > 0)))
        return MPPI_ERR_ARG;
    if (model->terrain != 0 && model->terrain != 1) return MPPI_ERR_ARG;
    if (model->n_static_boxes < 0 || model->n_static_boxes > MAX_SBOX) return MPPI_ERR_ARG;
    if (model->n_trunk_spheres < 0 || model->n_trunk_spheres > 4) return MPPI_ERR_ARG;
    if (cost->gait < 0 || cost->gait > 2 || (cost->gait == 2 && !(cost->raibert_len > 0))) return MPPI_ERR_ARG;
    if (model->terrain == 1 && mem_kind(model->hf, current_device()) == Mem::FOREIGN) return MPPI_ERR_ARG;

    mppi_handle h = new mppi_handle_s();
    h->model_in = *model;
    h->cost_in = *cost;
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    derive_model(*model, cfg->dt / cfg->n_sub, h->dm);
    derive_cost(*cost, h->dc);
    h->nx = h->dm.nx;
    h->D = cfg->interp == MPPI_INTERP_DIRECT ? NJ * cfg->H : D;
    const size_t K = (size_t)cfg->K, Dp = (size_t)h->D;
    auto al = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    bool ok = al((void**)&h->d_mu, Dp * sizeof(float)) && al((void**)&h->d_mu_prop, D * sizeof(float)) &&
              al((void**)&h->d_mu_upd, Dp * sizeof(float)) && al((void**)&h->d_U, K * Dp * sizeof(float)) &&
              al((void**)&h->d_L, K * sizeof(float)) && al((void**)&h->d_x0, K * NX_BOX * sizeof(float)) &&
              al((void**)&h->d_u0, NJ * sizeof(float)) && al((void**)&h->d_status, sizeof(int)) &&
              al((void**)&h->d_wsum, sizeof(double)) &&
              al((void**)&h->d_part, std::max({update_part_doubles((int)Dp), fused_part_doubles(*cfg),
                                                cfg->interp == MPPI_INTERP_DIRECT
                                                    ? update_direct_part_doubles((int)Dp) : (size_t)0}) *
                                         sizeof(double)) &&
              al((void**)&h->d_counter, update_counters((int)Dp) * sizeof(unsigned)) &&
              al((void**)&h->d_shard, 128 * sizeof(double)) &&
              al((void**)&h->d_B, (size_t)4 * cfg->H * sizeof(float));
    if (ok && model->terrain == 1) {
        size_t nh = (size_t)model->hf_nx * model->hf_ny;
        ok = al((void**)&h->d_hf, nh * sizeof(float));
        if (ok) {
            cudaMemcpyKind kind = is_device(model->hf) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            ok = cudaMemcpy(h->d_hf, model->hf, nh * sizeof(float), kind) == cudaSuccess;
        }
        h->dm.hf = h->d_hf;
    }
    if (ok) {
        float boxes[MAX_SBOX * 6] = {0};
        for (int i = 0; i < model->n_static_boxes; i++)
            for (int k = 0; k < 3; k++) {
                boxes[6 * i + k] = (float)model->sbox_lo[i][k];
                boxes[6 * i + 3 + k] = (float)model->sbox_hi[i][k];
            }
        memcpy(h->dm.sbox, boxes, sizeof(boxes));
        std::vector<float> heights;
        if (ok && model->terrain == 1) {
            heights.resize((size_t)model->hf_nx * model->hf_ny);
            ok = cudaMemcpy(heights.data(), h->d_hf, heights.size() * sizeof(float), cudaMemcpyDeviceToHost) ==
                 cudaSuccess;
        }
        h->model_key = model_key(h->dm, heights, boxes, MAX_SBOX * 6);
    }
    if (ok) {
        ok = cudaHostAlloc((void**)&h->h_box, BOX_FLOATS * sizeof(float), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostGetDevicePointer((void**)&h->d_box, h->h_box, 0) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    if (!ok) {
        mppi_destroy(h);
        return MPPI_ERR_OOM;
    }
    for (int i = 0; i < 4; i++) cudaEventCreate(&h->ev[i]);
    // default nominal: the cost's stand pose at every knot (every step for DIRECT)
    std::vector<float> mu0(Dp);
    for (size_t d = 0; d < Dp; d++) mu0[d] = (float)cost->stand[d % 3];
    std::vector<float> Bw;
    knot_weights(cfg->interp, cfg->H, Bw);
    if (cudaMemcpy(h->d_mu, mu0.data(), Dp * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_B, Bw.data(), Bw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->d_counter, 0, update_counters(h->D) * sizeof(unsigned)) != cudaSuccess) {
        mppi_destroy(h);
        return MPPI_ERR_CUDA;
    }
    *out = h;
    return MPPI_OK;
}

extern "C" mppi_status mppi_destroy(mppi_handle h) {
    if (!h) return MPPI_ERR_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    void* bufs[] = {h->d_mu,  h->d_mu_prop, h->d_mu_upd, h->d_U,    h->d_L,    h->d_x0,
                    h->d_u0,  h->d_hf,      h->d_status, h->d_wsum, h->d_part, h->d_counter,
                    h->d_B,      h->d_shard};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (h->h_box) cudaFreeHost(h->h_box);
    for (int i = 0; i < 4; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    delete h;
    return MPPI_OK;
}

extern "C" const char* mppi_last_error(mppi_handle h) { return h ? h->err.c_str() : "null handle"; }

extern "C" int mppi_state_size(mppi_handle h) { return h ? h->nx : 0; }

extern "C" int mppi_param_dim(mppi_handle h) { return h ? h->D : 0; }

extern "C" mppi_status mppi_set_nominal(mppi_handle h, const float* mu) {
    if (!h || !mu) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(mu);
    cudaMemcpyKind kind = is_device(mu) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h->d_mu, mu, (size_t)h->D * sizeof(float), kind, h->stream));
    if (kind == cudaMemcpyHostToDevice) CK(cudaStreamSynchronize(h->stream));
    return MPPI_OK;
}

extern "C" mppi_status mppi_get_nominal(mppi_handle h, float* mu_out) {
    if (!h || !mu_out) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(mu_out);
    bool dev = is_device(mu_out);
    CK(cudaMemcpyAsync(mu_out, h->d_mu, (size_t)h->D * sizeof(float),
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!dev) CK(cudaStreamSynchronize(h->stream));
    return MPPI_OK;
}

extern "C" mppi_status mppi_get_samples(mppi_handle h, float* U_out, float* L_out) {
    if (!h) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(U_out, L_out);
    const size_t K = (size_t)h->cfg.K;
    bool host = false;
    if (U_out) {
        const bool dev = is_device(U_out);
        host = host || !dev;
        CK(cudaMemcpyAsync(U_out, h->d_U, K * (size_t)h->D * sizeof(float),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    }
    if (L_out) {
        const bool dev = is_device(L_out);
        host = host || !dev;
        CK(cudaMemcpyAsync(L_out, h->d_L, K * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           h->stream));
    }
    if (host) CK(cudaStreamSynchronize(h->stream));
    return MPPI_OK;
}

static mppi_status do_sample(mppi_handle h, uint32_t step, const float* mu_prop, float* U) {
    SampleArgs a;
    a.mu = h->d_mu;
    a.mu_prop = nullptr;
    if (mu_prop) {
        const float* mp;
        mppi_status s = stage_in(h, mu_prop, D, h->d_mu_prop, &mp);
        if (s != MPPI_OK) return s;
        if (!aligned16(mp)) {  // the sampler reads the means as float4
            CK(cudaMemcpyAsync(h->d_mu_prop, mp, D * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
            mp = h->d_mu_prop;
        }
        a.mu_prop = mp;
    }
    a.U = U;
    memcpy(a.sigma, h->cfg.sigma, sizeof(a.sigma));
    memcpy(a.q_lo, h->cfg.q_lo, sizeof(a.q_lo));
    memcpy(a.q_hi, h->cfg.q_hi, sizeof(a.q_hi));
    a.key0 = (uint32_t)h->cfg.seed;
    a.key1 = (uint32_t)(h->cfg.seed >> 32);
    a.step = step;
    a.inst = h->cfg.inst;
    a.K = h->cfg.K;
    a.n_prop = h->cfg.n_prop;
    a.Dp = h->D;
    a.interp = h->cfg.interp;
    CK(launch_sample(a, h->stream));
    h->launches++;
    return MPPI_OK;
}

extern "C" mppi_status mppi_sample(mppi_handle h, uint32_t step, const float* mu_prop, float* U_out) {
    if (!h) return MPPI_ERR_ARG;
    LOCAL_CALL(mu_prop, U_out);
    bool host_out = U_out && !is_device(U_out);
    if (U_out && !host_out && !aligned16(U_out)) return fail(h, MPPI_ERR_ARG, "U_out must be 16-byte aligned");
    float* dst = (U_out && !host_out) ? U_out : h->d_U;
    mppi_status s = do_sample(h, step, mu_prop, dst);
    if (s != MPPI_OK) return s;
    if (host_out) {
        CK(cudaMemcpyAsync(U_out, h->d_U, (size_t)h->cfg.K * h->D * sizeof(float), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return MPPI_OK;
}

static RolloutArgs rollout_args(mppi_handle h, const float* x0, int per, const float* U, int n, double t0,
                                float* L, float* traj) {
    RolloutArgs a;
    a.model = h->dm;
    a.cost = h->dc;
    a.x0 = x0;
    a.x0_per_sample = per;
    a.U = U;
    a.L = L;
    a.traj = traj;
    a.n = n;
    a.H = h->cfg.H;
    a.n_sub = h->cfg.n_sub;
    a.dt = (float)h->cfg.dt;
    a.h = (float)(h->cfg.dt / h->cfg.n_sub);
    a.inv_Hm1 = (float)(1.0 / (h->cfg.H - 1));
    a.t0 = mppi_reduce_t0(h, t0);
    a.arm = (float)armature(h->model_in, h->cfg.dt / h->cfg.n_sub);
    a.Dp = h->D;
    a.interp = h->cfg.interp;
    a.Bt = reinterpret_cast<const float4*>(h->d_B);
    a.sample = 0;  // the knots come from U (mppi_step turns in-kernel sampling on)
    a.k_off = 0;
    a.mu = a.mu_prop = nullptr;
    a.K_all = h->cfg.K;
    a.n_prop = h->cfg.n_prop;
    memcpy(a.sigma, h->cfg.sigma, sizeof(a.sigma));
    memcpy(a.q_lo, h->cfg.q_lo, sizeof(a.q_lo));
    memcpy(a.q_hi, h->cfg.q_hi, sizeof(a.q_hi));
    a.key0 = (uint32_t)h->cfg.seed;
    a.key1 = (uint32_t)(h->cfg.seed >> 32);
    a.step = 0;
    a.inst = h->cfg.inst;
    a.U_out = nullptr;
    a.fuse = 0;  // mppi_step's knot representations fuse the update into the launch
    a.u0_host = a.mu_host = nullptr;
    a.status_host = nullptr;
    a.inv_lambda = 1.0 / (double)h->cfg.lambda;
    a.ctrl_steps = h->cfg.ctrl_steps;
    a.mu_w = nullptr;
    a.mu_upd = nullptr;
    a.u0 = nullptr;
    a.status = nullptr;
    a.wsum = nullptr;
    a.part = nullptr;
    a.counter = nullptr;
    return a;
}

static int rollout_block(mppi_handle h) { return rollout_block_cfg(h->cfg); }

extern "C" mppi_status mppi_rollouts(mppi_handle h, const float* x0, int x0_per_sample, const float* U, int n,
                                     double t0, float* L_out, float* traj_out) {
    if (!h || !x0 || n < 0) return fail(h, MPPI_ERR_ARG, "bad argument");
    LOCAL_CALL(x0, U, L_out, traj_out);
    const int nx = h->nx;
    const bool per = x0_per_sample != 0;
    if (!U && n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "n exceeds K for the handle's own samples");
    if (n == 0) return MPPI_OK;
    // x0
    const float* dx0;
    const size_t nx0 = (size_t)nx * (per ? n : 1);
    if (is_device(x0)) {
        dx0 = x0;
    } else {
        if (!all_finite(x0, nx0)) return fail(h, MPPI_ERR_NONFINITE, "x0 not finite");
        if (per && n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "host per-sample x0 limited to K states");
        CK(cudaMemcpyAsync(h->d_x0, x0, nx0 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        dx0 = h->d_x0;
    }
    // U
    const float* dU = h->d_U;
    if (U) {
        if (is_device(U)) {
            if (!aligned16(U)) return fail(h, MPPI_ERR_ARG, "U must be 16-byte aligned");
            dU = U;
        } else {
            if (n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "host U limited to K samples");
            CK(cudaMemcpyAsync(h->d_U, U, (size_t)n * h->D * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        }
    }
    // outputs
    float* dL = h->d_L;
    bool L_host = L_out && !is_device(L_out);
    if (L_out && !L_host) dL = L_out;
    if (!L_out || L_host)
        if (n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "host/internal L limited to K");
    float* dT = nullptr;
    bool T_host = traj_out && !is_device(traj_out);
    const size_t tbytes = (size_t)n * (h->cfg.H + 1) * nx * sizeof(float);
    if (traj_out) {
        if (T_host) CK(cudaMalloc(&dT, tbytes));
        else dT = traj_out;
    }
    RolloutArgs a = rollout_args(h, dx0, per, dU, n, t0, dL, dT);
    cudaError_t e = launch_rollout(a, rollout_block(h), h->stream);
    h->launches++;
    if (e != cudaSuccess) {
        if (T_host) cudaFree(dT);
        return cuda_fail(h, e, "rollout launch");
    }
    if (L_host) CK(cudaMemcpyAsync(L_out, dL, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (T_host) {
        cudaError_t e2 = cudaMemcpyAsync(traj_out, dT, tbytes, cudaMemcpyDeviceToHost, h->stream);
        cudaError_t e3 = cudaStreamSynchronize(h->stream);
        cudaFree(dT);
        if (e2 != cudaSuccess) return cuda_fail(h, e2, "traj copy");
        if (e3 != cudaSuccess) return cuda_fail(h, e3, "traj sync");
    } else if (L_host) {
        CK(cudaStreamSynchronize(h->stream));
    }
    return MPPI_OK;
}

static mppi_status do_update(mppi_handle h, const float* dL, const float* dU, int n) {
    UpdateArgs a;
    a.L = dL;
    a.U = dU;
    a.mu = h->d_mu;
    a.mu_upd = h->d_mu_upd;
    a.u0 = h->d_u0;
    a.status = h->d_status;
    a.wsum = h->d_wsum;
    a.part = h->d_part;
    a.counter = h->d_counter;
    a.n = n;
    a.H = h->cfg.H;
    a.ctrl_steps = h->cfg.ctrl_steps;
    a.inv_lambda = 1.0 / (double)h->cfg.lambda;
    a.Dp = h->D;
    a.interp = h->cfg.interp;
    a.partial_out = nullptr;
    CK(launch_update(a, h->stream));
    h->launches++;
    return MPPI_OK;
}

// copy the step's outputs (u0, mu before the shift) and read the status
// where the caller wants the outputs (u0_out / mu_out may be null)
struct OutPlace {
    bool u0_host = false, mu_host = false;
};
static OutPlace out_place(const float* u0_out, const float* mu_out) {
    OutPlace o;
    o.u0_host = u0_out && !is_device(u0_out);
    o.mu_host = mu_out && !is_device(mu_out);
    return o;
}

// device outputs are copied on the stream; host outputs come through a
// synchronisation, from the mailbox when the kernel wrote them there (boxed),
// else by copies from the device buffers
static mppi_status finish_outputs(mppi_handle h, float* u0_out, float* mu_out, const OutPlace& o, bool boxed) {
    if (u0_out && (!o.u0_host || !boxed))
        CK(cudaMemcpyAsync(u0_out, h->d_u0, NJ * sizeof(float),
                           o.u0_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    if (mu_out && (!o.mu_host || !boxed))
        CK(cudaMemcpyAsync(mu_out, h->d_mu_upd, (size_t)h->D * sizeof(float),
                           o.mu_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    if (o.u0_host || o.mu_host) {
        int st = 0;
        if (!boxed) CK(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (boxed) {
            const volatile float* box = h->h_box;
            if (o.u0_host)
                for (int i = 0; i < NJ; i++) u0_out[i] = box[BOX_U0 + i];
            if (o.mu_host)
                for (int i = 0; i < D; i++) mu_out[i] = box[BOX_MU + i];
            st = reinterpret_cast<const volatile int*>(box)[BOX_STATUS];
        }
        if (st != 0) return fail(h, MPPI_ERR_NONFINITE, "every rollout cost is non-finite; mean kept");
    }
    return MPPI_OK;
}
static mppi_status finish_outputs(mppi_handle h, float* u0_out, float* mu_out) {
    return finish_outputs(h, u0_out, mu_out, out_place(u0_out, mu_out), false);
}

extern "C" mppi_status mppi_update(mppi_handle h, const float* L, const float* U, int n, float* mu_out,
                                   float* u0_out) {
    if (!h || n < 0) return fail(h, MPPI_ERR_ARG, "bad argument");
    LOCAL_CALL(L, U, mu_out, u0_out);
    const float* dL = h->d_L;
    const float* dU = h->d_U;
    if ((!L || !U) && n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "n exceeds K");
    if (L) {
        if (!is_device(L) && n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "host L limited to K");
        mppi_status s = stage_in(h, L, (size_t)n, h->d_L, &dL);
        if (s != MPPI_OK) return s;
    }
    if (U) {
        if (is_device(U)) {
            if (!aligned16(U)) return fail(h, MPPI_ERR_ARG, "U must be 16-byte aligned");
            dU = U;
        } else {
            if (n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "host U limited to K");
            CK(cudaMemcpyAsync(h->d_U, U, (size_t)n * h->D * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        }
    }
    mppi_status s = do_update(h, dL, dU, n);
    if (s != MPPI_OK) return s;
    return finish_outputs(h, u0_out, mu_out);
}

extern "C" mppi_status mppi_step(mppi_handle h, const float* x0, uint32_t step, float* u0_out, float* mu_out) {
    if (!h || !x0) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(x0, u0_out, mu_out);
    const int nx = h->nx;
    const float* dx0;
    if (is_device(x0)) {
        dx0 = x0;
    } else {
        if (!all_finite(x0, nx)) return fail(h, MPPI_ERR_NONFINITE, "x0 not finite");
        CK(cudaMemcpyAsync(h->d_x0, x0, nx * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        dx0 = h->d_x0;
    }
    const bool tm = h->timing != 0;
    const bool knots = h->cfg.interp != MPPI_INTERP_DIRECT;
    if (tm) CK(cudaEventRecord(h->ev[0], h->stream));
    mppi_status s = MPPI_OK;
    // direct targets are sampled by K1; the knot forms sample inside the rollout kernel
    if (!knots) s = do_sample(h, step, nullptr, h->d_U);
    if (s != MPPI_OK) return s;
    if (tm) CK(cudaEventRecord(h->ev[1], h->stream));
    const double t0 = (double)step * h->cfg.ctrl_steps * h->cfg.dt;
    RolloutArgs a = rollout_args(h, dx0, 0, h->d_U, h->cfg.K, t0, h->d_L, nullptr);
    // Eq. 1, Eq. 2, apply and shift at the end of the same launch (grids of up to
    // FUSE_MAX_CTAS CTAs; larger ones run the update kernel after it)
    const bool fuse = knots && rollout_grid(h->cfg.K, rollout_block(h)) <= FUSE_MAX_CTAS;
    if (knots) {
        a.sample = 1;
        a.mu = h->d_mu;
        a.mu_prop = h->has_prop ? h->d_mu_prop : nullptr;
        a.step = step;
        a.U_out = h->d_U;
        a.fuse = fuse ? 1 : 0;
        a.mu_w = h->d_mu;
        a.mu_upd = h->d_mu_upd;
        a.u0 = h->d_u0;
        a.status = h->d_status;
        a.wsum = h->d_wsum;
        a.part = h->d_part;
        a.counter = h->d_counter;
    }
    // host-bound outputs of a fused step: the kernel writes them into the mailbox
    const OutPlace op = out_place(u0_out, mu_out);
    const bool boxed = fuse && (op.u0_host || op.mu_host);
    if (boxed) {
        a.u0_host = op.u0_host ? h->d_box + BOX_U0 : nullptr;
        a.mu_host = op.mu_host ? h->d_box + BOX_MU : nullptr;
        a.status_host = reinterpret_cast<int*>(h->d_box) + BOX_STATUS;
    }
    CK(launch_rollout(a, rollout_block(h), h->stream));
    h->launches++;
    if (tm) CK(cudaEventRecord(h->ev[2], h->stream));
    if (!fuse) {
        s = do_update(h, h->d_L, h->d_U, h->cfg.K);
        if (s != MPPI_OK) return s;
    }
    if (tm) {
        CK(cudaEventRecord(h->ev[3], h->stream));
        h->timed_valid = 1;
    }
    return finish_outputs(h, u0_out, mu_out, op, boxed);
}

// ---------------------------------------------------------------- sharded step

extern "C" mppi_status mppi_step_partial(mppi_handle h, const float* x0, uint32_t step, int k0, int n,
                                         double* part_out) {
    if (!h || !x0 || !part_out) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(x0, part_out);
    if (h->cfg.interp == MPPI_INTERP_DIRECT) return fail(h, MPPI_ERR_ARG, "sharded steps take the knot forms");
    if (k0 < 0 || n < 1 || (long)k0 + n > h->cfg.K) return fail(h, MPPI_ERR_ARG, "sample range outside 0..K");
    const float* dx0;
    if (is_device(x0)) {
        dx0 = x0;
    } else {
        if (!all_finite(x0, h->nx)) return fail(h, MPPI_ERR_NONFINITE, "x0 not finite");
        CK(cudaMemcpyAsync(h->d_x0, x0, h->nx * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        dx0 = h->d_x0;
    }
    // samples k0 .. k0 + n - 1 of the step, drawn in the rollout kernel at their
    // global indices and stored from row 0 of the handle's workspace
    const double t0 = (double)step * h->cfg.ctrl_steps * h->cfg.dt;
    RolloutArgs a = rollout_args(h, dx0, 0, h->d_U, n, t0, h->d_L, nullptr);
    a.sample = 1;
    a.k_off = k0;
    a.mu = h->d_mu;
    a.mu_prop = h->has_prop ? h->d_mu_prop : nullptr;
    a.step = step;
    a.U_out = h->d_U;
    CK(launch_rollout(a, rollout_block(h), h->stream));
    h->launches++;
    UpdateArgs u;
    u.L = h->d_L;
    u.U = h->d_U;
    u.mu = h->d_mu;
    u.mu_upd = h->d_mu_upd;
    u.u0 = h->d_u0;
    u.status = h->d_status;
    u.wsum = nullptr;
    u.part = h->d_part;
    u.counter = h->d_counter;
    u.n = n;
    u.H = h->cfg.H;
    u.ctrl_steps = h->cfg.ctrl_steps;
    u.inv_lambda = 1.0 / (double)h->cfg.lambda;
    u.Dp = D;
    u.interp = h->cfg.interp;
    u.partial_out = h->d_shard;
    CK(launch_update_partial(u, h->stream));
    h->launches++;
    const bool dev = is_device(part_out);
    CK(cudaMemcpyAsync(part_out, h->d_shard, MPPI_SHARD_PARTIAL * sizeof(double),
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!dev) CK(cudaStreamSynchronize(h->stream));
    return MPPI_OK;
}

extern "C" mppi_status mppi_step_finalize(mppi_handle h, const double* sums, float* u0_out, float* mu_out) {
    if (!h || !sums) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(sums, u0_out, mu_out);
    if (h->cfg.interp == MPPI_INTERP_DIRECT) return fail(h, MPPI_ERR_ARG, "sharded steps take the knot forms");
    const double* ds = h->d_shard + 64;
    if (is_device(sums)) {
        ds = sums;
    } else {
        CK(cudaMemcpyAsync(h->d_shard + 64, sums, (MPPI_SHARD_PARTIAL - 1) * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
    }
    FinalizeArgs f;
    f.sums = ds;
    f.mu = h->d_mu;
    f.mu_upd = h->d_mu_upd;
    f.u0 = h->d_u0;
    f.status = h->d_status;
    f.H = h->cfg.H;
    f.ctrl_steps = h->cfg.ctrl_steps;
    f.interp = h->cfg.interp;
    CK(launch_update_finalize(f, h->stream));
    h->launches++;
    return finish_outputs(h, u0_out, mu_out);
}

extern "C" mppi_status mppi_step_proposal(mppi_handle h, mppi_mlp net, const float* x0, uint32_t step, float* u0_out,
                                          float* mu_out) {
    if (!h || !net || !x0) return fail(h, MPPI_ERR_ARG, "null argument");
    LOCAL_CALL(x0, u0_out, mu_out);
    if (mppi_mlp_device(net) != h->device) return fail(h, MPPI_ERR_ARG, "the network lives on another device");
    if (h->cfg.n_prop < 1) return fail(h, MPPI_ERR_ARG, "the handle was created with n_prop = 0");
    if (h->cfg.interp == MPPI_INTERP_DIRECT) return fail(h, MPPI_ERR_ARG, "the proposal is a knot mean");
    const int nx = h->nx;
    const float* dx0;
    if (is_device(x0)) {
        dx0 = x0;
    } else {
        if (!all_finite(x0, nx)) return fail(h, MPPI_ERR_NONFINITE, "x0 not finite");
        CK(cudaMemcpyAsync(h->d_x0, x0, nx * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        dx0 = h->d_x0;
    }
    // the network's forward on the features of x0 (computed in its kernel)
    // straight into the handle's proposal mean, then the step: two launches on
    // the handle's stream
    CK(mppi_mlp_forward_states_dev(net, dx0, nx, 1, mppi_feature_params(h, step), h->d_mu_prop, h->stream));
    h->launches++;
    h->has_prop = 1;
    return mppi_step(h, dx0, step, u0_out, mu_out);
}

extern "C" mppi_status mppi_selftest_noise_tables(float* radius, float* cosv, float* sinv, void* stream) {
    if (!radius || !cosv || !sinv || !is_device(radius) || !is_device(cosv) || !is_device(sinv)) return MPPI_ERR_ARG;
    return launch_noise_tables(radius, cosv, sinv, (cudaStream_t)stream) == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

extern "C" mppi_status mppi_set_timing(mppi_handle h, int on) {
    if (!h) return MPPI_ERR_ARG;
    h->timing = on;
    h->timed_valid = 0;
    return MPPI_OK;
}

extern "C" mppi_status mppi_get_timings(mppi_handle h, float ms[3]) {
    if (!h || !ms) return fail(h, MPPI_ERR_ARG, "null argument");
    if (!h->timed_valid) return fail(h, MPPI_ERR_ARG, "no timed step yet (mppi_set_timing first)");
    CK(cudaEventSynchronize(h->ev[3]));
    for (int i = 0; i < 3; i++) CK(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
    return MPPI_OK;
}

extern "C" mppi_status mppi_launch_count(mppi_handle h, uint64_t* count) {
    if (!h || !count) return MPPI_ERR_ARG;
    *count = h->launches;
    return MPPI_OK;
}
