// handle.h -- the controller handle behind the C ABI (internal to the library;
// shared by api.cu and the multi-instance code in batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mppi.h"
#include "features.cuh"
#include "kernels.h"

// the mailbox's layout (floats): u0, mu', status (an int)
constexpr int BOX_U0 = 0, BOX_MU = mppi::NJ, BOX_STATUS = mppi::NJ + mppi::D, BOX_FLOATS = 64;

struct mppi_handle_s {
    mppi_model_t model_in;
    mppi_cost_t cost_in;
    mppi_config_t cfg;
    mppi::DevModel dm;
    mppi::DevCost dc;
    uint64_t model_key = 0;  // hash of dm's values, heights and static boxes (equal keys: the same model)
    cudaStream_t stream = nullptr;
    int device = 0;
    int nx = mppi::NX_ROBOT;
    int D = mppi::D;  // parameters per sample: 48, or 12 H for direct targets
    float *d_mu = nullptr, *d_mu_prop = nullptr, *d_mu_upd = nullptr, *d_U = nullptr, *d_L = nullptr;
    float *d_x0 = nullptr, *d_u0 = nullptr, *d_hf = nullptr;
    float* d_B = nullptr;  // [H][4] knot weights of each dt step (16-B aligned rows)
    int* d_status = nullptr;
    // pinned, device-mapped mailbox: u0 [12], mu' [48], status; the control
    // step's kernel writes host-bound outputs here (no device-to-host copies)
    float* h_box = nullptr;
    float* d_box = nullptr;  // its device address
    double* d_wsum = nullptr;
    double* d_part = nullptr;      // update scratch: per-CTA partial sums
    double* d_shard = nullptr;     // sharded step: [64] a shard's partial sums, [64] the combined sums
    unsigned* d_counter = nullptr;  // update scratch: finished-CTA counter
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int timing = 0;
    int has_prop = 0;  // mppi_step samples the last n_prop samples around d_mu_prop
    int timed_valid = 0;
    uint64_t launches = 0;
    std::string err;
};


// internal launchers shared by the units (no host synchronisation)
// what the proposal network's features take besides the state, for this handle at control index `step`
mppi::FeatParams mppi_feature_params(mppi_handle h, uint32_t step);
// the device the network's buffers live on
int mppi_mlp_device(mppi_mlp net);
// the network's small-batch forward: n <= 128 device rows dX [n][62] -> dY [n][48]
cudaError_t mppi_mlp_forward_small_dev(mppi_mlp net, const float* dX, int n, float* dY, cudaStream_t st);
// the same on the features (features.cuh) of n device states dS (row stride lds),
// computed inside the forward's kernel
cudaError_t mppi_mlp_forward_states_dev(mppi_mlp net, const float* dS, int lds, int n, const mppi::FeatParams& fp,
                                        float* dY, cudaStream_t st);

// implicit-PD armature of one sub-step: h (kd + h kp) + a0
double mppi_armature(const mppi_model_t& p, double h);
// gait time of a horizon starting at absolute time t0, reduced modulo the gait period
float mppi_reduce_t0(const mppi_handle h, double t0);
