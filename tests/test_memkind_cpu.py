"""CPU check of the C ABI's buffer classification (csrc/memkind.h): which
caller buffers a call on the current device uses in place, which it stages
through a copy, and which it rejects -- device memory of another GPU -- with no
GPU present.  The header is compiled by the host compiler against a stand-in
for the CUDA runtime's pointer-attribute query, whose answers the test sets."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the three runtime calls memkind.h makes, answered from a table the program fills
FAKE_RUNTIME = r'''
#pragma once
enum cudaError_t { cudaSuccess = 0, cudaErrorInvalidValue = 1 };
enum cudaMemoryType { cudaMemoryTypeUnregistered = 0, cudaMemoryTypeHost = 1, cudaMemoryTypeDevice = 2,
                      cudaMemoryTypeManaged = 3 };
struct cudaPointerAttributes { cudaMemoryType type; int device; void* devicePointer; void* hostPointer; };
struct FakePtr { const void* p; int known; cudaMemoryType type; int device; };
extern FakePtr g_fake[16];
extern int g_nfake, g_current, g_errors_cleared;
inline cudaError_t cudaGetDevice(int* d) { *d = g_current; return g_current < 0 ? cudaErrorInvalidValue : cudaSuccess; }
inline cudaError_t cudaGetLastError() { g_errors_cleared++; return cudaSuccess; }
inline cudaError_t cudaPointerGetAttributes(cudaPointerAttributes* a, const void* p) {
    for (int i = 0; i < g_nfake; i++)
        if (g_fake[i].p == p) {
            if (!g_fake[i].known) return cudaErrorInvalidValue;
            a->type = g_fake[i].type;
            a->device = g_fake[i].device;
            return cudaSuccess;
        }
    a->type = cudaMemoryTypeUnregistered;
    a->device = -2;
    return cudaSuccess;
}
'''

SRC = r'''
#include <cstdio>
#include "cuda_runtime.h"
#include "memkind.h"
using namespace mppi;
FakePtr g_fake[16];
int g_nfake = 0, g_current = 0, g_errors_cleared = 0;
static char buf[8];
static const char* name(Mem m) {
    return m == Mem::NONE ? "none" : m == Mem::HOST ? "host" : m == Mem::LOCAL ? "local" : "foreign";
}
int main() {
    // buf + 0: device memory of GPU 0; + 1: of GPU 1; + 2: managed (reported on GPU 1);
    // + 3: pinned host; + 4: unregistered host; + 5: a pointer the query rejects
    g_fake[0] = {buf + 0, 1, cudaMemoryTypeDevice, 0};
    g_fake[1] = {buf + 1, 1, cudaMemoryTypeDevice, 1};
    g_fake[2] = {buf + 2, 1, cudaMemoryTypeManaged, 1};
    g_fake[3] = {buf + 3, 1, cudaMemoryTypeHost, 0};
    g_fake[4] = {buf + 4, 1, cudaMemoryTypeUnregistered, -2};
    g_fake[5] = {buf + 5, 0, cudaMemoryTypeUnregistered, 0};
    g_nfake = 6;
    for (int dev = 0; dev < 2; dev++) {
        g_current = dev;
        printf("dev%d", dev);
        printf(" %s", name(mem_kind(nullptr, dev)));
        for (int i = 0; i < 6; i++) printf(" %s", name(mem_kind(buf + i, dev)));
        printf(" |");
        for (int i = 0; i < 6; i++) printf(" %d", (int)is_local(buf + i));
        printf(" | %d %d %d", (int)any_foreign(dev, {buf + 0, buf + 3, nullptr}),
               (int)any_foreign(dev, {buf + 2, buf + 4, buf + 5}), (int)any_foreign(dev, {buf + 1}));
        printf(" |");
        for (int i = 0; i < 6; i++) printf(" %d", (int)host_accessible(buf + i));
        printf("\n");
    }
    g_current = -1;  // the runtime cannot name a device: no device memory is local (managed still is)
    printf("nodev %d %d %d\n", current_device(), (int)is_local(buf + 0), (int)is_local(buf + 2));
    printf("cleared %d\n", g_errors_cleared);
    return 0;
}
'''


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("memkind")
    (d / "cuda_runtime.h").write_text(FAKE_RUNTIME)
    (d / "main.cpp").write_text(SRC)
    exe = d / "memkind"
    subprocess.run([cxx, "-std=c++17", "-Wall", "-Werror", "-I", str(d),
                    "-I", os.path.join(ROOT, "paper_2409_10469_gb300", "csrc"),
                    str(d / "main.cpp"), "-o", str(exe)], check=True, capture_output=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()


def test_classification_per_current_device(lines):
    # order: null, GPU-0 memory, GPU-1 memory, managed, pinned host, plain host, unknown
    assert lines[0].split("|")[0].split() == ["dev0", "none", "local", "foreign", "local", "host", "host", "host"]
    assert lines[1].split("|")[0].split() == ["dev1", "none", "foreign", "local", "local", "host", "host", "host"]
    assert lines[0].split("|")[1].split() == ["1", "0", "1", "0", "0", "0"]
    assert lines[1].split("|")[1].split() == ["0", "1", "1", "0", "0", "0"]


def test_another_gpus_memory_is_flagged(lines):
    # any_foreign: (GPU 0, pinned, null), (managed, host, unknown), (GPU 1)
    assert lines[0].split("|")[2].split() == ["0", "0", "1"]
    assert lines[1].split("|")[2].split() == ["1", "0", "0"]


def test_host_access_excludes_plain_device_memory(lines):
    for ln in lines[:2]:
        assert ln.split("|")[3].split() == ["0", "0", "1", "1", "1", "1"]


def test_no_current_device_and_error_state_cleared(lines):
    assert lines[2].split() == ["nodev", "-1", "0", "1"]
    # the rejected queries (the unknown pointer, the failed device query) clear
    # the runtime's error state
    assert int(lines[3].split()[1]) > 0
