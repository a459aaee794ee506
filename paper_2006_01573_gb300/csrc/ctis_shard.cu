// The ratio step of a wavelength-sharded EM iteration (Eqs. 2 and 8).
//
// H f = sum_s H_s f_s: a rank that owns the wavelengths of a slice forms the
// partial image of its slice, the ranks' partials are summed (the caller's
// all-reduce), and every rank then needs u = g / (H f) for its own adjoint
// and update. The windowed forward's fused ratio epilogue sees only the local
// partial, so this step is a kernel of its own: u into the FPA copies the
// adjoint reads, and the statistics of the iterate (the same four sums as the
// fused path, over the support of H f) in a fixed order.
#include <cuda_runtime.h>

#include "ctis_internal.h"
#include "ctis_kernels.h"

namespace ctis {
namespace {

constexpr int kRatioThreads = 256;
constexpr int kRatioBlocks = 1024;

__device__ __forceinline__ float warp_sum32(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// u = g / q where q > 0 (else 0) into `ncopies` x-shifted copies (copy c holds
// column x at x + c); per block the float32 sums of each thread's pixels,
// added over the warp in float32 and over the block's warps in float64 in
// warp order, into part[block][kNumStats].
__global__ void __launch_bounds__(kRatioThreads)
    ratio_stats_kernel(float* copies, long long copy_stride, int ncopies, int pitch, const float* q,
                       const float* g, int width, int height, double* part) {
    __shared__ double ws[kRatioThreads / 32][kNumStats];
    const long long n = (long long)width * height;
    float st[kNumStats] = {0.f, 0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % width);
        const long long y = i / width;
        const float qv = q[i], gv = g[i];
        float u = 0.f;
        if (qv > 0.f) {
            u = gv / qv;
            st[0] += qv;
            st[1] += gv;
            st[2] += gv * logf(qv) - qv;
            const float d = gv - qv;
            st[3] += d * d;
        }
        float* d = copies + y * pitch + x;
        for (int c = 0; c < ncopies; ++c) d[c * copy_stride + c] = u;
    }
    if (!part) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) {
        const float s = warp_sum32(st[k]);
        if (lane == 0) ws[warp][k] = static_cast<double>(s);
    }
    __syncthreads();
    if (threadIdx.x < kNumStats) {
        double t = ws[0][threadIdx.x];
        for (int w = 1; w < kRatioThreads / 32; ++w) t += ws[w][threadIdx.x];
        part[(long long)blockIdx.x * kNumStats + threadIdx.x] = t;
    }
}

constexpr int kFinishThreads = 256;
constexpr int kFinishGroups = kFinishThreads / kNumStats;   // 64 groups per statistic

// out[k] = sum over the blocks of part[block][k] in a fixed order: group j of
// statistic k adds blocks j, j + 64, j + 128, ... in turn, then the 64 group
// sums are added pairwise in a fixed tree (same result on every run).
__global__ void __launch_bounds__(kFinishThreads)
    stats_finish_kernel(const double* part, int blocks, double* out) {
    __shared__ double gs[kFinishGroups][kNumStats];
    const int k = threadIdx.x % kNumStats, j = threadIdx.x / kNumStats;
    double t = 0.0;
    for (int b = j; b < blocks; b += kFinishGroups) t += part[(long long)b * kNumStats + k];
    gs[j][k] = t;
    __syncthreads();
    for (int half = kFinishGroups / 2; half > 0; half >>= 1) {
        if (j < half) gs[j][k] += gs[j + half][k];
        __syncthreads();
    }
    if (j == 0) out[k] = gs[0][k];
}

}  // namespace

int shard_ratio_blocks() { return kRatioBlocks; }

cudaError_t launch_shard_ratio(float* copies, long long copy_stride, int ncopies, int pitch,
                               const float* q, const float* g, int width, int height, double* part,
                               double* stats_out, cudaStream_t stream) {
    ratio_stats_kernel<<<kRatioBlocks, kRatioThreads, 0, stream>>>(
        copies, copy_stride, ncopies, pitch, q, g, width, height, stats_out ? part : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !stats_out) return e;
    stats_finish_kernel<<<1, kFinishThreads, 0, stream>>>(part, kRatioBlocks, stats_out);
    return cudaGetLastError();
}

}  // namespace ctis
