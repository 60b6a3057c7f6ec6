// batch.cu -- many MPPI instances in one persistent launch per control step.
//
// Each instance is a controller handle (its own model, cost, K, H, nominal and
// buffers).  One control step of a batch runs Alg. 1 of arXiv 2409.10469
// (sample, roll out, weight by Eq. 1, update by Eq. 2, apply, shift) for every
// active instance in a single persistent kernel:
//   - the work is a list of items (instance, first sample, count), one item per
//     chunk of blockDim/4 rollouts, longest horizons first (so that the uneven
//     H of the instances does not leave a long tail);
//   - blocks (a grid of blocks_per_sm x SMs) take items from an atomic counter
//     until the list is exhausted -- no block ever waits on another;
//   - an item samples its knots in-kernel (the same Philox/Box-Muller code and
//     clamp as the sampling kernel, so the knots are bit-identical), rolls them
//     out with the same per-lane simulator as the single-instance kernel, and
//     writes U and L;
//   - the block that completes an instance's last chunk (an atomic count of
//     finished samples per instance reaches K) runs that instance's update in
//     one block, in a fixed order, so an instance's result does not depend on
//     which other instances share the launch.
// When all instances share one model and one cost (equal model keys: the
// values, heights and boxes hash alike), the launch passes them in the kernel's
// parameters and a specialisation reads them there, as the single-instance
// kernel does, instead of from each item's shared-memory descriptor.
// The host side captures [work-list copy, step indices, counter resets, kernel]
// in a CUDA graph once per block shape; the autotuner times the candidate block
// shapes on the batch itself and keeps the fastest.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "batch.cuh"
#include "batch_kernel.cuh"
#include "handle.h"
#include "memkind.h"

using namespace mppi;

namespace mppi {

// the shared-model kernels are compiled in batch_uni.cu (no box) and batch_uni_box.cu
#define MPPI_UNI_EXTERN(B)                                                                  \
    extern template cudaError_t launch_k_batch<B, UNI_FLAT>(const BatchArgs&, int, cudaStream_t);    \
    extern template cudaError_t launch_k_batch<B, UNI_TERRAIN>(const BatchArgs&, int, cudaStream_t); \
    extern template cudaError_t launch_k_batch<B, UNI_FLAT_BOX>(const BatchArgs&, int, cudaStream_t); \
    extern template cudaError_t launch_k_batch<B, UNI_TERRAIN_BOX>(const BatchArgs&, int, cudaStream_t);
MPPI_UNI_EXTERN(64)
MPPI_UNI_EXTERN(128)
MPPI_UNI_EXTERN(256)
#undef MPPI_UNI_EXTERN

template <int BLOCK>
static cudaError_t launch_batch_t(const BatchArgs& a, int grid, cudaStream_t st) {
    if (!a.uniform) return launch_k_batch<BLOCK, UNI_NONE>(a, grid, st);
    switch (uni_kind(a.model)) {
        case UNI_FLAT: return launch_k_batch<BLOCK, UNI_FLAT>(a, grid, st);
        case UNI_TERRAIN: return launch_k_batch<BLOCK, UNI_TERRAIN>(a, grid, st);
        case UNI_FLAT_BOX: return launch_k_batch<BLOCK, UNI_FLAT_BOX>(a, grid, st);
        default: return launch_k_batch<BLOCK, UNI_TERRAIN_BOX>(a, grid, st);
    }
}

void set_uniform(BatchArgs& a, const InstDesc* d, int n) {
    a.uniform = n > 0;
    for (int i = 1; i < n && a.uniform; i++)
        a.uniform = d[i].model_key == d[0].model_key && memcmp(&d[i].cost, &d[0].cost, sizeof(DevCost)) == 0;
    if (a.uniform) {
        a.model = d[0].model;
        a.cost = d[0].cost;
    } else {
        memset(&a.model, 0, sizeof(a.model));
        memset(&a.cost, 0, sizeof(a.cost));
    }
}

cudaError_t launch_batch(const BatchArgs& a, int block, int grid, cudaStream_t st) {
    switch (block) {
        case 64: return launch_batch_t<64>(a, grid, st);
        case 128: return launch_batch_t<128>(a, grid, st);
        case 256: return launch_batch_t<256>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int max_blocks_per_sm(int block) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    // (every variant has the same launch bounds)
    if (block == 64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<64, UNI_NONE>, 64, 0);
    if (block == 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<128, UNI_NONE>, 128, 0);
    if (block == 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<256, UNI_NONE>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace mppi

// ------------------------------------------------------------------ host side

struct mppi_batch_s {
    std::vector<mppi_handle> hs;
    int n = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    int block = 128, blocks_per_sm = 4;
    int max_items = 0;
    std::vector<InstDesc> h_desc;  // host copies of the descriptors (the uniform-model test)
    InstDesc* d_desc = nullptr;
    WorkItem* d_items = nullptr;
    int *d_nitems = nullptr, *d_next = nullptr;
    unsigned* d_done = nullptr;
    float *d_x0s = nullptr, *d_u0s = nullptr;
    uint32_t* d_steps = nullptr;
    WorkItem* h_items = nullptr;  // pinned
    int* h_nitems = nullptr;      // pinned
    uint32_t* h_steps = nullptr;  // pinned
    float *h_x0s = nullptr, *h_u0s = nullptr;  // pinned
    cudaGraphExec_t exec = nullptr;
    int graph_block = 0, graph_bpsm = 0;
    int device = 0;  // every handle's and the batch's buffers live here
    uint64_t launches = 0;
    std::string err;
};

static mppi_status bfail(mppi_batch b, mppi_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}
#define BCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return bfail(b, MPPI_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// memory of the current device (or managed memory)
static bool dev_ptr(const void* p) { return is_local(p); }

// the batch's device is the current one and no buffer is another GPU's memory
static mppi_status local_call(mppi_batch b, std::initializer_list<const void*> bufs) {
    const int dev = current_device();
    if (dev < 0) return bfail(b, MPPI_ERR_CUDA, "cudaGetDevice failed");
    if (dev != b->device) return bfail(b, MPPI_ERR_ARG, "the batch's device is not the current device");
    if (any_foreign(dev, bufs)) return bfail(b, MPPI_ERR_ARG, "a buffer is memory of another GPU");
    return MPPI_OK;
}

InstDesc mppi::make_desc(const mppi_handle_s* h) {
    InstDesc d;
    memset(&d, 0, sizeof(d));
    d.model = h->dm;
    d.cost = h->dc;
    d.mu = h->d_mu;
    d.mu_upd = h->d_mu_upd;
    d.u0 = h->d_u0;
    d.U = h->d_U;
    d.L = h->d_L;
    d.status = h->d_status;
    d.mu_prop = h->cfg.n_prop > 0 ? h->d_mu_prop : nullptr;  // filled by mppi_set_proposal
    d.K = h->cfg.K;
    d.H = h->cfg.H;
    d.n_sub = h->cfg.n_sub;
    d.n_prop = h->cfg.n_prop;
    d.ctrl_steps = h->cfg.ctrl_steps;
    d.nx = h->nx;
    d.gait = h->cost_in.gait;
    d.h = (float)(h->cfg.dt / h->cfg.n_sub);
    d.dt = (float)h->cfg.dt;
    d.inv_Hm1 = (float)(1.0 / (h->cfg.H - 1));
    d.arm = (float)mppi_armature(h->model_in, h->cfg.dt / h->cfg.n_sub);
    d.inv_lambda = 1.0 / (double)h->cfg.lambda;
    d.dt_d = h->cfg.dt;
    d.period_d = h->cost_in.gait_period;
    d.interp = h->cfg.interp;
    d.Bt = reinterpret_cast<const float4*>(h->d_B);
    d.model_key = h->model_key;
    memcpy(d.sigma, h->cfg.sigma, sizeof(d.sigma));
    memcpy(d.q_lo, h->cfg.q_lo, sizeof(d.q_lo));
    memcpy(d.q_hi, h->cfg.q_hi, sizeof(d.q_hi));
    d.key0 = (uint32_t)h->cfg.seed;
    d.key1 = (uint32_t)(h->cfg.seed >> 32);
    d.inst_id = h->cfg.inst;
    return d;
}

// work list of the active instances, longest horizons first
static int build_items(mppi_batch b, const int* active) {
    const int R = b->block / 4;
    std::vector<int> order;
    for (int i = 0; i < b->n; i++)
        if (!active || active[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const long cx = (long)b->hs[x]->cfg.H * b->hs[x]->cfg.n_sub, cy = (long)b->hs[y]->cfg.H * b->hs[y]->cfg.n_sub;
        return cx > cy;
    });
    int n = 0;
    for (int i : order)
        for (int k0 = 0; k0 < b->hs[i]->cfg.K; k0 += R) {
            WorkItem w = {i, k0, std::min(R, b->hs[i]->cfg.K - k0)};
            b->h_items[n++] = w;
        }
    *b->h_nitems = n;
    return n;
}

// the step's device work: copy the work list and step indices, reset the
// counters, run the persistent kernel
static cudaError_t enqueue_step(mppi_batch b) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_items, b->h_items, (size_t)b->max_items * sizeof(WorkItem), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(b->d_nitems, b->h_nitems, sizeof(int), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(b->d_steps, b->h_steps, (size_t)b->n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->d_next, 0, sizeof(int), b->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->d_done, 0, (size_t)b->n * sizeof(unsigned), b->stream)) != cudaSuccess) return e;
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.desc = b->d_desc;
    a.items = b->d_items;
    a.n_items = b->d_nitems;
    a.next = b->d_next;
    a.done = b->d_done;
    a.x0s = b->d_x0s;
    a.steps = b->d_steps;
    a.u0s = b->d_u0s;
    set_uniform(a, b->h_desc.data(), b->n);
    return launch_batch(a, b->block, b->blocks_per_sm * b->sms, b->stream);
}

static mppi_status rebuild_graph(mppi_batch b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t cap;
    BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = b->stream;
    b->stream = cap;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = enqueue_step(b);
        e = cudaStreamEndCapture(cap, &g);
        if (e1 != cudaSuccess) e = e1;
    }
    b->stream = saved;
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->exec = nullptr;
        return bfail(b, MPPI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->graph_block = b->block;
    b->graph_bpsm = b->blocks_per_sm;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_create(const mppi_handle* hs, int n, void* stream, mppi_batch* out) {
    if (!hs || n < 1 || !out) return MPPI_ERR_ARG;
    *out = nullptr;
    mppi_batch b = new mppi_batch_s();
    b->n = n;
    b->stream = (cudaStream_t)stream;
    const int dev = current_device();
    b->device = dev;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<InstDesc> descs;
    int max_items = 0;
    for (int i = 0; i < n; i++) {
        // batches run the knot representations of handles on the current device
        if (!hs[i] || hs[i]->cfg.interp == MPPI_INTERP_DIRECT || hs[i]->device != dev) {
            delete b;
            return MPPI_ERR_ARG;
        }
        b->hs.push_back(hs[i]);
        descs.push_back(make_desc(hs[i]));
        max_items += (hs[i]->cfg.K + 15) / 16;  // enough for the smallest block shape (64 threads)
    }
    b->max_items = max_items;
    b->h_desc = descs;
    bool ok = cudaMalloc((void**)&b->d_desc, n * sizeof(InstDesc)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_items, max_items * sizeof(WorkItem)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_nitems, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_next, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_done, n * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_x0s, (size_t)n * NX_BOX * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_u0s, (size_t)n * NJ * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&b->d_steps, n * sizeof(uint32_t)) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_items, max_items * sizeof(WorkItem)) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_nitems, sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_steps, n * sizeof(uint32_t)) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_x0s, (size_t)n * NX_BOX * sizeof(float)) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_u0s, (size_t)n * NJ * sizeof(float)) == cudaSuccess;
    if (!ok || cudaMemcpy(b->d_desc, descs.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_done, 0, n * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b->d_x0s, 0, (size_t)n * NX_BOX * sizeof(float)) != cudaSuccess ||
        cudaMemset(b->d_u0s, 0, (size_t)n * NJ * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        mppi_batch_destroy(b);
        return MPPI_ERR_OOM;
    }
    memset(b->h_items, 0, max_items * sizeof(WorkItem));
    memset(b->h_steps, 0, n * sizeof(uint32_t));
    b->block = 128;
    b->blocks_per_sm = std::max(1, std::min(4, max_blocks_per_sm(128)));
    *out = b;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_destroy(mppi_batch b) {
    if (!b) return MPPI_ERR_ARG;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    void* d[] = {b->d_desc, b->d_items, b->d_nitems, b->d_next, b->d_done, b->d_x0s, b->d_u0s, b->d_steps};
    for (void* p : d)
        if (p) cudaFree(p);
    void* hp[] = {b->h_items, b->h_nitems, b->h_steps, b->h_x0s, b->h_u0s};
    for (void* p : hp)
        if (p) cudaFreeHost(p);
    delete b;
    return MPPI_OK;
}

extern "C" const char* mppi_batch_last_error(mppi_batch b) { return b ? b->err.c_str() : "null batch"; }

extern "C" mppi_status mppi_batch_set_shape(mppi_batch b, int block, int blocks_per_sm) {
    if (!b) return MPPI_ERR_ARG;
    if (block != 64 && block != 128 && block != 256) return bfail(b, MPPI_ERR_ARG, "block must be 64, 128 or 256");
    const int mx = max_blocks_per_sm(block);
    if (blocks_per_sm < 1 || blocks_per_sm > mx)
        return bfail(b, MPPI_ERR_ARG, "blocks_per_sm out of range (occupancy limit " + std::to_string(mx) + ")");
    b->block = block;
    b->blocks_per_sm = blocks_per_sm;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_get_shape(mppi_batch b, int* block, int* blocks_per_sm) {
    if (!b || !block || !blocks_per_sm) return MPPI_ERR_ARG;
    *block = b->block;
    *blocks_per_sm = b->blocks_per_sm;
    return MPPI_OK;
}

// stage x0s (host or device, [n][NX_BOX]) and step indices (host, [n]) for the next step
static mppi_status stage_inputs(mppi_batch b, const float* x0s, const uint32_t* steps) {
    if (steps) memcpy(b->h_steps, steps, (size_t)b->n * sizeof(uint32_t));
    if (x0s) {
        if (dev_ptr(x0s)) {
            BCK(cudaMemcpyAsync(b->d_x0s, x0s, (size_t)b->n * NX_BOX * sizeof(float), cudaMemcpyDeviceToDevice,
                                b->stream));
        } else {
            for (int i = 0; i < b->n * NX_BOX; i++)
                if (!isfinite(x0s[i])) return bfail(b, MPPI_ERR_NONFINITE, "x0s not finite");
            memcpy(b->h_x0s, x0s, (size_t)b->n * NX_BOX * sizeof(float));
            BCK(cudaMemcpyAsync(b->d_x0s, b->h_x0s, (size_t)b->n * NX_BOX * sizeof(float), cudaMemcpyHostToDevice,
                                b->stream));
        }
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_step(mppi_batch b, const int* active, const float* x0s, const uint32_t* steps,
                                       float* u0s) {
    if (!b) return MPPI_ERR_ARG;
    mppi_status s = local_call(b, {x0s, u0s});
    if (s != MPPI_OK) return s;
    s = stage_inputs(b, x0s, steps);
    if (s != MPPI_OK) return s;
    // the previous graph launch may still read the pinned work list: order the rewrite after it
    BCK(cudaStreamSynchronize(b->stream));
    build_items(b, active);
    if (!b->exec || b->graph_block != b->block || b->graph_bpsm != b->blocks_per_sm) {
        s = rebuild_graph(b);
        if (s != MPPI_OK) return s;
    }
    BCK(cudaGraphLaunch(b->exec, b->stream));
    b->launches++;
    if (u0s) {
        const bool dev = dev_ptr(u0s);
        if (dev) {
            BCK(cudaMemcpyAsync(u0s, b->d_u0s, (size_t)b->n * NJ * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
        } else {
            BCK(cudaMemcpyAsync(b->h_u0s, b->d_u0s, (size_t)b->n * NJ * sizeof(float), cudaMemcpyDeviceToHost,
                                b->stream));
            BCK(cudaStreamSynchronize(b->stream));
            memcpy(u0s, b->h_u0s, (size_t)b->n * NJ * sizeof(float));
        }
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_autotune(mppi_batch b, const float* x0s, int trials, int* block_out,
                                           int* bpsm_out, float* best_ms_out) {
    if (!b || trials < 1) return MPPI_ERR_ARG;
    mppi_status s = local_call(b, {x0s});
    if (s != MPPI_OK) return s;
    s = stage_inputs(b, x0s, nullptr);
    if (s != MPPI_OK) return s;
    // every candidate starts from the same nominals: save them, restore after each trial
    std::vector<float*> saved(b->n, nullptr);
    for (int i = 0; i < b->n; i++) {
        BCK(cudaMalloc((void**)&saved[i], D * sizeof(float)));
        BCK(cudaMemcpyAsync(saved[i], b->hs[i]->d_mu, D * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
    }
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_b = b->block, best_p = b->blocks_per_sm;
    const int blocks[3] = {64, 128, 256};
    for (int bi = 0; bi < 3; bi++) {
        const int mx = max_blocks_per_sm(blocks[bi]);
        for (int p = 1; p <= mx && p <= 16; p++) {  // every occupancy level up to the limit
            b->block = blocks[bi];
            b->blocks_per_sm = p;
            BCK(cudaStreamSynchronize(b->stream));
            build_items(b, nullptr);
            float tot = 0.f;
            for (int t = 0; t <= trials; t++) {
                for (int i = 0; i < b->n; i++)
                    BCK(cudaMemcpyAsync(b->hs[i]->d_mu, saved[i], D * sizeof(float), cudaMemcpyDeviceToDevice,
                                        b->stream));
                BCK(cudaEventRecord(e0, b->stream));
                BCK(enqueue_step(b));
                BCK(cudaEventRecord(e1, b->stream));
                BCK(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, e0, e1));
                if (t > 0) tot += ms;  // the first run warms up
            }
            const float mean = tot / trials;
            if (mean < best) {
                best = mean;
                best_b = blocks[bi];
                best_p = p;
            }
        }
    }
    for (int i = 0; i < b->n; i++) {
        BCK(cudaMemcpyAsync(b->hs[i]->d_mu, saved[i], D * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    for (float* p : saved) cudaFree(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->block = best_b;
    b->blocks_per_sm = best_p;
    if (block_out) *block_out = best_b;
    if (bpsm_out) *bpsm_out = best_p;
    if (best_ms_out) *best_ms_out = best;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_launch_count(mppi_batch b, uint64_t* count) {
    if (!b || !count) return MPPI_ERR_ARG;
    *count = b->launches;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_shared_model(mppi_batch b, int* shared) {
    if (!b || !shared) return MPPI_ERR_ARG;
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    set_uniform(a, b->h_desc.data(), b->n);
    *shared = a.uniform;
    return MPPI_OK;
}

extern "C" mppi_status mppi_batch_get_means(mppi_batch b, float* mu_upds, float* nominals) {
    if (!b) return MPPI_ERR_ARG;
    const mppi_status s = local_call(b, {mu_upds, nominals});
    if (s != MPPI_OK) return s;
    const bool hu = mu_upds && !dev_ptr(mu_upds), hn = nominals && !dev_ptr(nominals);
    for (int i = 0; i < b->n; i++) {
        if (mu_upds)
            BCK(cudaMemcpyAsync(mu_upds + (size_t)i * D, b->hs[i]->d_mu_upd, D * sizeof(float),
                                hu ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
        if (nominals)
            BCK(cudaMemcpyAsync(nominals + (size_t)i * D, b->hs[i]->d_mu, D * sizeof(float),
                                hn ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
    }
    if (hu || hn) BCK(cudaStreamSynchronize(b->stream));
    return MPPI_OK;
}
