// memkind.h -- where a caller's buffer lives, for the C ABI's argument checks.
//
// Every call runs its kernels and copies on the current device.  A caller's
// buffer may be host memory (pageable, pinned or registered: staged through a
// copy) or memory of that device (used in place; managed memory counts as
// such).  Device memory of another GPU is neither: a kernel would reach it
// through a peer mapping that need not exist, so the entry points reject it as
// an argument error instead of faulting.
#pragma once
#include <cuda_runtime.h>

#include <initializer_list>

namespace mppi {

enum class Mem { NONE, HOST, LOCAL, FOREIGN };

// the current device, or -1 when the runtime cannot say
inline int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}

// p classified for a call on device dev (NONE for a null pointer)
inline Mem mem_kind(const void* p, int dev) {
    if (!p) return Mem::NONE;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // not known to the runtime: plain host memory
        return Mem::HOST;
    }
    if (at.type == cudaMemoryTypeManaged) return Mem::LOCAL;
    if (at.type == cudaMemoryTypeDevice) return at.device == dev ? Mem::LOCAL : Mem::FOREIGN;
    return Mem::HOST;
}

// memory the host may read and write directly: host memory of any kind, or
// managed memory (plain device memory is not)
inline bool host_accessible(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type != cudaMemoryTypeDevice;
}

// device memory of the current device (or managed memory)
inline bool is_local(const void* p) { return mem_kind(p, current_device()) == Mem::LOCAL; }

// true when any of the pointers is device memory of a GPU other than dev
inline bool any_foreign(int dev, std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (mem_kind(p, dev) == Mem::FOREIGN) return true;
    return false;
}

}  // namespace mppi
