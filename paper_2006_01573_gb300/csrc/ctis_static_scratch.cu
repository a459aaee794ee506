// Fixed, library-owned scratch for ctis_forward_static_scratch.
//
// Some callers cannot call cudaMalloc when they project: real-time loops that
// forbid allocation after start-up, code that has handed all device memory to
// its own pool or arena, or code running while a stream is captured into a
// CUDA graph in a mode that rejects allocation. For them the forward
// projection can take its scratch from this array instead of the plan's
// workspace. The array lives in the library's device image, so every GPU
// that loads the library holds it (kStaticScratchBytes) until the process
// exits.
#include <cuda_runtime.h>

#include <mutex>

#include "ctis_kernels.h"

namespace ctis {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

}  // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }

// Device address of the array on the current device. The first call on a
// device looks the symbol up (with that device current) and caches it; the
// host-side name g_static_scratch is not a device address and must never be
// passed to a kernel.
cudaError_t static_scratch_ptr(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace ctis
