// serve.cu -- serving runtime: continuous batching of MPPI control-step
// requests from many robots on one GPU.
//
// A robot is a controller handle: its model, cost, K, H and its nominal knots
// stay on the device between requests (device-resident controller state).  A
// request asks for one control step of one robot from a state x0.  The
// runtime
//   - queues requests (one outstanding request per robot: its nominal is
//     updated in place by the step);
//   - admits them by memory: a solve needs K x 49 floats of workspace (knots
//     and costs), carved first-fit from one device pool whose size is the
//     memory budget; the queue is served in arrival order and admission stops
//     at the first request that does not fit, so a large solve is never
//     starved by smaller ones behind it;
//   - launches the admitted requests together as one persistent multi-instance
//     step (the kernel of batch.cu) on one of two launch contexts, each with
//     its own stream, so that requests admitted while another launch is still
//     on the GPU run concurrently with it;
//   - retires a launch when its completion event has fired: copies each
//     robot's control out, frees the workspace, stamps the latency (arrival to
//     observed completion on the host clock).
// Every result is computed by the same per-instance arithmetic whatever else is
// in the launch (see batch.cu), so a robot's control is identical alone and in
// the mix.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "batch.cuh"
#include "handle.h"
#include "memkind.h"

using namespace mppi;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// first-fit allocator over [0, size) with coalescing frees
struct Pool {
    size_t size = 0, in_use = 0, peak = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t s) {
        size = s;
        free_.clear();
        free_[0] = s;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, o = it->first + n;
                free_.erase(it);
                if (rest) free_[o] = rest;
                in_use += n;
                peak = std::max(peak, in_use);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        in_use -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Request {
    int robot;
    uint32_t step;
    float x0[NX_BOX];
    double t_arrive;
    size_t ws_off = 0, ws_len = 0;
};

struct Robot {
    mppi_handle h;
    InstDesc tmpl;
    size_t ws_bytes;
    bool outstanding = false;  // a request is queued or in flight
    bool ready = false;        // a result waits to be polled
    float u0[NJ];
    double latency = 0;
};

struct Launch {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    std::vector<Request> reqs;
    InstDesc *d_desc = nullptr, *h_desc = nullptr;
    WorkItem *d_items = nullptr, *h_items = nullptr;
    int *d_nitems = nullptr, *h_nitems = nullptr, *d_next = nullptr;
    unsigned* d_done = nullptr;
    float *d_x0s = nullptr, *h_x0s = nullptr, *d_u0s = nullptr, *h_u0s = nullptr;
    uint32_t *d_steps = nullptr, *h_steps = nullptr;
};

}  // namespace

struct mppi_server_s {
    char* d_pool = nullptr;
    Pool pool;
    int max_robots = 0, max_items = 0;
    std::vector<Robot> robots;
    std::deque<Request> queue;
    Launch L[2];
    int block = 128, bpsm = 2, sms = 0;
    int device = 0;  // the robots' handles and the server's buffers live here
    uint64_t submitted = 0, completed = 0, launches = 0, busy_rejects = 0;
    double rollout_steps = 0;
    std::vector<double> lat;
    std::string err;
};

static mppi_status sfail(mppi_server s, mppi_status st, const std::string& m) {
    if (s) s->err = m;
    return st;
}
#define SCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return sfail(s, MPPI_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

extern "C" mppi_status mppi_server_create(size_t budget_bytes, int max_robots, int max_samples, mppi_server* out) {
    if (!out || budget_bytes < ALIGN || max_robots < 1 || max_samples < 1) return MPPI_ERR_ARG;
    *out = nullptr;
    mppi_server s = new mppi_server_s();
    s->max_robots = max_robots;
    // enough work items for max_robots solves of max_samples at 16 rollouts per item
    s->max_items = max_robots * ((max_samples + 15) / 16);
    const int dev = current_device();
    s->device = dev;
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    s->bpsm = std::max(1, std::min(2, max_blocks_per_sm(s->block)));
    bool ok = cudaMalloc((void**)&s->d_pool, budget_bytes) == cudaSuccess;
    for (int i = 0; ok && i < 2; i++) {
        Launch& l = s->L[i];
        ok = cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc((void**)&l.d_desc, max_robots * sizeof(InstDesc)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_desc, max_robots * sizeof(InstDesc)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_items, s->max_items * sizeof(WorkItem)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_items, s->max_items * sizeof(WorkItem)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_nitems, sizeof(int)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_nitems, sizeof(int)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_next, sizeof(int)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_done, max_robots * sizeof(unsigned)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_x0s, (size_t)max_robots * NX_BOX * sizeof(float)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_x0s, (size_t)max_robots * NX_BOX * sizeof(float)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_u0s, (size_t)max_robots * NJ * sizeof(float)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_u0s, (size_t)max_robots * NJ * sizeof(float)) == cudaSuccess &&
             cudaMalloc((void**)&l.d_steps, max_robots * sizeof(uint32_t)) == cudaSuccess &&
             cudaMallocHost((void**)&l.h_steps, max_robots * sizeof(uint32_t)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        mppi_server_destroy(s);
        return MPPI_ERR_OOM;
    }
    s->pool.init(budget_bytes);
    *out = s;
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_destroy(mppi_server s) {
    if (!s) return MPPI_ERR_ARG;
    for (Launch& l : s->L) {
        if (l.st) cudaStreamSynchronize(l.st);
        void* d[] = {l.d_desc, l.d_items, l.d_nitems, l.d_next, l.d_done, l.d_x0s, l.d_u0s, l.d_steps};
        for (void* p : d)
            if (p) cudaFree(p);
        void* hp[] = {l.h_desc, l.h_items, l.h_nitems, l.h_x0s, l.h_u0s, l.h_steps};
        for (void* p : hp)
            if (p) cudaFreeHost(p);
        if (l.ev) cudaEventDestroy(l.ev);
        if (l.st) cudaStreamDestroy(l.st);
    }
    if (s->d_pool) cudaFree(s->d_pool);
    delete s;
    return MPPI_OK;
}

extern "C" const char* mppi_server_last_error(mppi_server s) { return s ? s->err.c_str() : "null server"; }

extern "C" mppi_status mppi_server_add_robot(mppi_server s, mppi_handle h, int* robot_id) {
    if (!s || !h || !robot_id) return MPPI_ERR_ARG;
    if (h->cfg.interp == MPPI_INTERP_DIRECT) return sfail(s, MPPI_ERR_ARG, "served robots use a knot representation");
    if (h->device != s->device) return sfail(s, MPPI_ERR_ARG, "the handle lives on another device than the server");
    if ((int)s->robots.size() >= s->max_robots) return sfail(s, MPPI_ERR_ARG, "max_robots reached");
    if (h->cfg.K > (s->max_items / s->max_robots) * 16) return sfail(s, MPPI_ERR_ARG, "K above max_samples");
    Robot r;
    r.h = h;
    r.tmpl = make_desc(h);
    r.ws_bytes = align_up((size_t)h->cfg.K * D * sizeof(float)) + align_up((size_t)h->cfg.K * sizeof(float));
    if (r.ws_bytes > s->pool.size) return sfail(s, MPPI_ERR_ARG, "one solve of this robot exceeds the memory budget");
    memset(r.u0, 0, sizeof(r.u0));
    *robot_id = (int)s->robots.size();
    s->robots.push_back(r);
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_submit(mppi_server s, int robot, const float* x0, uint32_t step) {
    if (!s || !x0 || robot < 0 || robot >= (int)s->robots.size()) return MPPI_ERR_ARG;
    if (!host_accessible(x0)) return sfail(s, MPPI_ERR_ARG, "x0 must be host memory");
    Robot& r = s->robots[robot];
    if (r.outstanding) {
        s->busy_rejects++;
        return sfail(s, MPPI_ERR_BUSY, "robot has a request in progress");
    }
    Request q;
    q.robot = robot;
    q.step = step;
    memset(q.x0, 0, sizeof(q.x0));
    for (int i = 0; i < r.h->nx; i++) {
        if (!isfinite(x0[i])) return sfail(s, MPPI_ERR_NONFINITE, "x0 not finite");
        q.x0[i] = x0[i];
    }
    q.t_arrive = now_s();
    r.outstanding = true;
    r.ready = false;
    s->queue.push_back(q);
    s->submitted++;
    return MPPI_OK;
}

// retire a finished launch
static void retire(mppi_server s, Launch& l) {
    const double t = now_s();
    for (size_t i = 0; i < l.reqs.size(); i++) {
        const Request& q = l.reqs[i];
        Robot& r = s->robots[q.robot];
        memcpy(r.u0, l.h_u0s + i * NJ, sizeof(r.u0));
        r.latency = t - q.t_arrive;
        r.ready = true;
        r.outstanding = false;
        s->pool.release(q.ws_off, q.ws_len);
        s->lat.push_back(r.latency);
        s->completed++;
        s->rollout_steps += (double)r.h->cfg.K * r.h->cfg.H;
    }
    l.reqs.clear();
    l.in_flight = false;
}

// admit queued requests into launch l (arrival order, stop at the first that
// does not fit the pool) and launch them; returns how many were admitted
static int admit_and_launch(mppi_server s, Launch& l, mppi_status* st) {
    *st = MPPI_OK;
    int n = 0;
    while (!s->queue.empty() && n < s->max_robots) {
        Request q = s->queue.front();
        Robot& r = s->robots[q.robot];
        size_t off;
        if (!s->pool.alloc(r.ws_bytes, &off)) break;
        s->queue.pop_front();
        q.ws_off = off;
        q.ws_len = r.ws_bytes;
        InstDesc d = r.tmpl;
        d.U = (float*)(s->d_pool + off);
        d.L = (float*)(s->d_pool + off + align_up((size_t)r.h->cfg.K * D * sizeof(float)));
        l.h_desc[n] = d;
        memcpy(l.h_x0s + (size_t)n * NX_BOX, q.x0, sizeof(q.x0));
        l.h_steps[n] = q.step;
        l.reqs.push_back(q);
        n++;
    }
    if (n == 0) return 0;
    // block shape: a set sharing one model runs the parameter-bank kernel at the
    // server's shape; a mixed set runs the general kernel at 256 threads, one
    // block per SM, where it needs no spill (at 128 threads it spills to local
    // memory; on the 64-robot mix 256 x 1 is the autotuner's choice)
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    set_uniform(a, l.h_desc, n);
    const int block = a.uniform ? s->block : 256;
    const int bpsm = a.uniform ? s->bpsm : 1;
    const int R = block / 4;
    // work items, longest horizons first
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long)l.h_desc[a].H * l.h_desc[a].n_sub > (long)l.h_desc[b].H * l.h_desc[b].n_sub;
    });
    int ni = 0;
    for (int i : order)
        for (int k0 = 0; k0 < l.h_desc[i].K; k0 += R) l.h_items[ni++] = WorkItem{i, k0, std::min(R, l.h_desc[i].K - k0)};
    *l.h_nitems = ni;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    ok(cudaMemcpyAsync(l.d_desc, l.h_desc, n * sizeof(InstDesc), cudaMemcpyHostToDevice, l.st));
    ok(cudaMemcpyAsync(l.d_items, l.h_items, ni * sizeof(WorkItem), cudaMemcpyHostToDevice, l.st));
    ok(cudaMemcpyAsync(l.d_nitems, l.h_nitems, sizeof(int), cudaMemcpyHostToDevice, l.st));
    ok(cudaMemcpyAsync(l.d_x0s, l.h_x0s, (size_t)n * NX_BOX * sizeof(float), cudaMemcpyHostToDevice, l.st));
    ok(cudaMemcpyAsync(l.d_steps, l.h_steps, n * sizeof(uint32_t), cudaMemcpyHostToDevice, l.st));
    ok(cudaMemsetAsync(l.d_next, 0, sizeof(int), l.st));
    ok(cudaMemsetAsync(l.d_done, 0, n * sizeof(unsigned), l.st));
    a.desc = l.d_desc;
    a.items = l.d_items;
    a.n_items = l.d_nitems;
    a.next = l.d_next;
    a.done = l.d_done;
    a.x0s = l.d_x0s;
    a.steps = l.d_steps;
    a.u0s = l.d_u0s;
    ok(launch_batch(a, block, bpsm * s->sms, l.st));
    ok(cudaMemcpyAsync(l.h_u0s, l.d_u0s, (size_t)n * NJ * sizeof(float), cudaMemcpyDeviceToHost, l.st));
    ok(cudaEventRecord(l.ev, l.st));
    if (e != cudaSuccess) {
        *st = sfail(s, MPPI_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        return n;
    }
    l.in_flight = true;
    s->launches++;
    return n;
}

extern "C" mppi_status mppi_server_tick(mppi_server s, int* completed_out) {
    if (!s) return MPPI_ERR_ARG;
    int done = 0;
    for (Launch& l : s->L)
        if (l.in_flight) {
            cudaError_t q = cudaEventQuery(l.ev);
            if (q == cudaSuccess) {
                done += (int)l.reqs.size();
                retire(s, l);
            } else if (q != cudaErrorNotReady) {
                return sfail(s, MPPI_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(q));
            }
        }
    for (Launch& l : s->L)
        if (!l.in_flight && !s->queue.empty()) {
            mppi_status st;
            admit_and_launch(s, l, &st);
            if (st != MPPI_OK) return st;
        }
    if (completed_out) *completed_out = done;
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_poll(mppi_server s, int robot, float* u0_out, double* latency_s, int* ready) {
    if (!s || robot < 0 || robot >= (int)s->robots.size() || !ready) return MPPI_ERR_ARG;
    if (u0_out && !host_accessible(u0_out)) return sfail(s, MPPI_ERR_ARG, "u0_out must be host memory");
    Robot& r = s->robots[robot];
    *ready = r.ready ? 1 : 0;
    if (r.ready) {
        if (u0_out) memcpy(u0_out, r.u0, sizeof(r.u0));
        if (latency_s) *latency_s = r.latency;
        r.ready = false;
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_stats(mppi_server s, mppi_server_stats_t* o) {
    if (!s || !o) return MPPI_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->launches = s->launches;
    o->busy_rejects = s->busy_rejects;
    o->queued = (uint64_t)s->queue.size();
    o->in_flight = (uint64_t)(s->L[0].reqs.size() + s->L[1].reqs.size());
    o->pool_bytes = s->pool.size;
    o->pool_in_use = s->pool.in_use;
    o->pool_peak = s->pool.peak;
    o->rollout_steps = s->rollout_steps;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        o->latency_p50 = pct(0.50);
        o->latency_p99 = pct(0.99);
        o->latency_max = v.back();
    }
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_reset_stats(mppi_server s) {
    if (!s) return MPPI_ERR_ARG;
    s->lat.clear();
    s->completed = s->submitted = s->launches = s->busy_rejects = 0;
    s->rollout_steps = 0;
    s->pool.peak = s->pool.in_use;
    return MPPI_OK;
}

extern "C" mppi_status mppi_server_drain(mppi_server s) {
    if (!s) return MPPI_ERR_ARG;
    while (!s->queue.empty() || s->L[0].in_flight || s->L[1].in_flight) {
        for (Launch& l : s->L)
            if (l.in_flight) SCK(cudaEventSynchronize(l.ev));
        mppi_status st = mppi_server_tick(s, nullptr);
        if (st != MPPI_OK) return st;
    }
    return MPPI_OK;
}
