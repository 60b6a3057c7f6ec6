// noalloc.cu -- mppi_update_noalloc: the Eq. 1 / Eq. 2 update with its scratch
// memory in a fixed device array instead of a handle's allocations.
//
// Who needs this: code that runs where allocating device memory is not an
// option -- a real-time control thread that must never block in the driver's
// allocator, a process whose memory pool is owned by another framework, an
// embedded runtime that forbids cudaMalloc after start-up, or a library call
// made while another component holds the allocator.  Such a caller still owns
// and passes every input and output buffer; the only memory this call adds is
// the file-scope array below, which every GPU that loads the library keeps for
// the life of the process.
//
// The update kernel needs per-CTA partial sums and a finished-CTA counter.  Here
// they live in `g_update_scratch` (51,456 bytes: a row of 50 doubles -- 48 sums,
// the weight sum and the chunk's cost minimum -- for each of the at most 128
// CTAs, and a 256-byte slot for the counter).  n only sets how many samples each
// of those CTAs sums, so no n up to MPPI_NOALLOC_MAX_N needs more scratch.  Host
// code cannot use the symbol itself as a device address: on each device the
// first call asks the runtime for the array's address (cudaGetSymbolAddress,
// with that device current) and caches it.  That first call should therefore
// happen before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mppi.h"
#include "kernels.h"
#include "memkind.h"

using namespace mppi;

namespace {

constexpr size_t PART_DOUBLES = update_part_doubles(D);
constexpr size_t SCRATCH_BYTES = PART_DOUBLES * sizeof(double) + 256;  // partials + counter slot

static_assert(SCRATCH_BYTES == 51456, "the scratch size stated in include/mppi.h");
static_assert(PART_DOUBLES == (size_t)UPDATE_MAX_CTAS * (D + 2), "one row per CTA of the clamped grid");

static __device__ __align__(256) unsigned char g_update_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {nullptr};

// device memory of GPU `dev` (or managed memory): the kernels run on the current
// device, so a buffer on another GPU is rejected instead of being reached
// through a peer mapping that may not exist
bool on_device(const void* p, int dev) { return mem_kind(p, dev) == Mem::LOCAL; }

}  // namespace

extern "C" mppi_status mppi_update_noalloc(const float* L, const float* U, int n, int H, int ctrl_steps,
                                           double lambda, int interp, const float* mu_in, float* mu_out,
                                           float* mu_upd_out, float* u0_out, int* status_out, void* stream) {
    if (n < 1 || n > MPPI_NOALLOC_MAX_N || H < 2 || ctrl_steps < 1 || !(lambda > 0)) return MPPI_ERR_ARG;
    // the knot representations (48 parameters); direct targets need 12 H
    if (interp != MPPI_INTERP_CUBIC && interp != MPPI_INTERP_ZERO && interp != MPPI_INTERP_LINEAR)
        return MPPI_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MPPI_ERR_CUDA;
    if (!on_device(L, dev) || !on_device(U, dev) || !on_device(mu_in, dev) || !on_device(mu_out, dev) ||
        !on_device(u0_out, dev))
        return MPPI_ERR_ARG;
    if ((mu_upd_out && !on_device(mu_upd_out, dev)) || (status_out && !on_device(status_out, dev)))
        return MPPI_ERR_ARG;
    if (((uintptr_t)U & 15u) != 0) return MPPI_ERR_ARG;

    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_update_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return MPPI_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)base;
    unsigned* counter = (unsigned*)((unsigned char*)base + PART_DOUBLES * sizeof(double));
    // the counter must read zero when the kernel starts; the partials need no clearing
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess) return MPPI_ERR_CUDA;
    if (mu_out != mu_in &&
        cudaMemcpyAsync(mu_out, mu_in, D * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MPPI_ERR_CUDA;

    UpdateArgs a;
    a.L = L;
    a.U = U;
    a.mu = mu_out;
    a.mu_upd = mu_upd_out;
    a.u0 = u0_out;
    a.status = status_out;
    a.wsum = nullptr;
    a.part = part;
    a.counter = counter;
    a.n = n;
    a.H = H;
    a.ctrl_steps = ctrl_steps;
    a.inv_lambda = 1.0 / lambda;
    a.Dp = D;                 // a knot representation: 48 parameters
    a.interp = interp;        // MPPI_INTERP_* equals the kernels' INTERP_* (api.cu checks it)
    a.partial_out = nullptr;
    return launch_update(a, st) == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}
