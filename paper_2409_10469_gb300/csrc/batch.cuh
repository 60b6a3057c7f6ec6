// batch.cuh -- the persistent multi-instance step shared by batches (batch.cu)
// and the serving runtime (serve.cu): per-instance descriptors, work items and
// the launch entry point of the persistent kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct mppi_handle_s;

namespace mppi {

struct InstDesc {
    DevModel model;
    DevCost cost;
    float* mu;            // nominal knots, updated in place (shifted)
    float* mu_upd;        // updated mean before the shift
    float* u0;            // applied control
    float* U;             // [K][48] sampled knots
    float* L;             // [K] costs
    int* status;          // 0 ok, 4 all costs non-finite
    const float* mu_prop; // proposal mean or null
    int K, H, n_sub, n_prop, ctrl_steps, nx, gait;
    float h, dt, inv_Hm1, arm;
    double inv_lambda;    // 1 / lambda (the weights' exponent is formed in FP64)
    double dt_d, period_d;
    float sigma[D], q_lo[3], q_hi[3];
    uint32_t key0, key1, inst_id;
    int interp;           // MPPI_INTERP_* (knot representations only)
    const float4* Bt;     // [H] knot weights of each dt step
    uint64_t model_key;   // the handle's model key (equal keys: the same model values)
};

struct WorkItem {
    int inst, k0, n;
};

struct BatchArgs {
    const InstDesc* desc;
    const WorkItem* items;
    const int* n_items;
    int* next;
    unsigned* done;
    const float* x0s;       // [n_inst][NX_BOX]
    const uint32_t* steps;  // [n_inst] control-step index of each instance
    float* u0s;             // [n_inst][12]
    // when every instance of the launch has the same model and cost (set_uniform),
    // the kernel reads them from here -- the parameter bank, whose words the
    // arithmetic takes as operands -- instead of each item's shared-memory copy
    int uniform;
    DevModel model;
    DevCost cost;
};

// fill the uniform fields of a launch over descriptors d[0 .. n)
void set_uniform(BatchArgs& a, const InstDesc* d, int n);

// launch the persistent kernel (block in {64, 128, 256}; grid = blocks_per_sm x SMs)
cudaError_t launch_batch(const BatchArgs& a, int block, int grid, cudaStream_t st);
// occupancy limit of the persistent kernel for a block size (0 if unsupported)
int max_blocks_per_sm(int block);
// descriptor of a controller handle; U / L point at the handle's own workspace
InstDesc make_desc(const mppi_handle_s* h);

}  // namespace mppi
