// FP32 FMA-pipe microbenchmark: the measured ceiling of the projectors'
// roofline. The projectors are bound by float32 fused multiply-adds (the
// gather evaluates nnz(H) of them per projection), so their roofline is the
// rate at which this GPU retires independent FFMAs. Each thread keeps kChains
// independent accumulation chains in registers (no memory traffic in the
// loop) and advances each by four FMAs per iteration; the packed form issues
// the same work as FFMA2 pairs. The result goes to `out` so the chains are
// not optimised away.
#include <cuda_runtime.h>

#include "ctis.h"

namespace {

constexpr int kChains = 8;

__global__ void fma_peak_scalar(int iters, float* out, float seed) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed + 1e-7f * float(threadIdx.x + 31 * i);
    const float b = 0.99999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma_peak_packed(int iters, float* out, float seed) {
    float2 a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i)
        a[i] = make_float2(seed + 1e-7f * float(threadIdx.x + 31 * i), seed - 1e-7f * float(i));
    const float2 b = make_float2(0.99999f, 0.99998f), c = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int ctis_fma_peak(int packed, int blocks, int threads, int iters, float* out_dev,
                             void* stream) {
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 || !out_dev)
        return CTIS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (packed)
        fma_peak_packed<<<blocks, threads, 0, st>>>(iters, out_dev, 1.0f);
    else
        fma_peak_scalar<<<blocks, threads, 0, st>>>(iters, out_dev, 1.0f);
    return cudaGetLastError() == cudaSuccess ? CTIS_OK : CTIS_ERR_CUDA;
}
