// Host-side dispatch of the gather projectors, their geometry queries, and the
// small data-movement kernels around them (x-shifted copies in and out, the
// Sec. 3 index map).
#include "ctis_gather.cuh"

namespace ctis {

cudaError_t gather_prepare_fwd(int K, int dtype, int shape, int* blocks_per_sm);
cudaError_t gather_launch_fwd(int K, int dtype, int shape, const CUtensorMap& win,
                              const GatherParams& p, cudaStream_t stream);
cudaError_t gather_prepare_adj(int K, int dtype, int* blocks_per_sm);
cudaError_t gather_launch_adj(int K, int dtype, const CUtensorMap& win, const GatherParams& p,
                              cudaStream_t stream);
#ifdef CTIS_DEBUG_BOUNDS
cudaError_t debug_arm_fwd(const DbgRanges& r);
cudaError_t debug_arm_adj(const DbgRanges& r);
#endif

namespace {

// ---------------------------------------------------------------------------
// small utility kernels
// ---------------------------------------------------------------------------
// Writes the NC x-shifted copies of a plane stack: copy q, element x + q, is
// src[x] (or `value` when src is null); the other elements of a copy's row
// stay as they are (zero from the allocation).
template <typename T, typename TS>
__global__ void scatter_copies_kernel(T* dst, long long copy_stride, int ncopies, int dst_pitch,
                                      long long dst_plane_stride, const TS* src, int src_pitch,
                                      long long src_plane_stride, int width, int height,
                                      int planes, float value) {
    const long long n = (long long)width * height * planes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % width);
        const long long r = i / width;
        const int y = int(r % height);
        const int z = int(r / height);
        const float v = src ? Elem<TS>::load(src + z * src_plane_stride + (long long)y * src_pitch + x)
                            : value;
        T* d = dst + z * dst_plane_stride + (long long)y * dst_pitch + x;
        for (int q = 0; q < ncopies; ++q) Elem<T>::store(d + q * copy_stride + q, v);
    }
}

// Copies copy 0 of a plane stack back to a dense caller buffer.
template <typename T>
__global__ void gather_copy0_kernel(T* dst, const T* src, int src_pitch, long long src_plane_stride,
                                    int width, int height, int planes) {
    const long long n = (long long)width * height * planes;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % width);
        const long long r = i / width;
        const int y = int(r % height);
        const int z = int(r / height);
        dst[i] = src[z * src_plane_stride + (long long)y * src_pitch + x];
    }
}

// ---- frames of a batch (device arrays of per-frame pointers) -------------
// dst[f * n + i] = srcs[f][i]
__global__ void frames_gather_kernel(float* dst, const float* const* srcs, long long n, int frames) {
    const long long total = n * frames;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = int(i / n);
        dst[i] = srcs[f][i - (long long)f * n];
    }
}

// x-shifted copies of every frame's datacube: plane f * planes + z of the copies
// receives srcs[f][z] (dense width x height planes), or `value` when srcs is null.
template <typename T>
__global__ void frames_scatter_copies_kernel(T* dst, long long copy_stride, int ncopies, int dst_pitch,
                                             long long dst_plane_stride, const T* const* srcs,
                                             float value, int width, int height, int planes,
                                             int frames) {
    const long long per_frame = (long long)width * height * planes;
    const long long total = per_frame * frames;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = int(i / per_frame);
        const long long j = i - (long long)f * per_frame;
        const int x = int(j % width);
        const long long r = j / width;
        const int y = int(r % height);
        const long long z = r / height;
        const float v = srcs ? Elem<T>::load(srcs[f] + j) : value;
        T* d = dst + ((long long)f * planes + z) * dst_plane_stride + (long long)y * dst_pitch + x;
        for (int q = 0; q < ncopies; ++q) Elem<T>::store(d + q * copy_stride + q, v);
    }
}

// copy 0 of every frame's datacube back to its dense buffer dsts[f]
template <typename T>
__global__ void frames_copy0_out_kernel(T* const* dsts, const T* src, int src_pitch,
                                        long long src_plane_stride, int width, int height,
                                        int planes, int frames) {
    const long long per_frame = (long long)width * height * planes;
    const long long total = per_frame * frames;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = int(i / per_frame);
        const long long j = i - (long long)f * per_frame;
        const int x = int(j % width);
        const long long r = j / width;
        const int y = int(r % height);
        const long long z = r / height;
        dsts[f][j] = src[((long long)f * planes + z) * src_plane_stride + (long long)y * src_pitch + x];
    }
}

// dst row gid[f] <- src row f (rows of `len` doubles)
__global__ void rows_scatter_kernel(double* dst, const double* src, const int* gid, int len,
                                    int frames) {
    const long long total = (long long)len * frames;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = int(i / len);
        const int e = int(i - (long long)f * len);
        dst[(long long)gid[f] * len + e] = src[i];
    }
}

// Frame totals of the forward's tile statistics when no following launch
// adds them: kStatSlices warps per frame.
__global__ void stats_reduce_kernel(double* out, const double* tile_stats, int tiles, int frames,
                                    long long frame_stride, double* part, int* tickets) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= frames * kStatSlices) return;
    const int f = r / kStatSlices;
    reduce_frame_slice(tile_stats, tiles, f, r - f * kStatSlices, part, tickets,
                       out + f * frame_stride, threadIdx.x & 31);
}

// Sec. 3 embedding: datacube element j = (p, r, s) sits at FPA pixel
// (x, y) = (p, r) of the s-th stacked FPA vector.
__device__ __forceinline__ long long stacked_fpa_index(int p, int r, int s, int gamma, long long n) {
    return (long long)p + (long long)gamma * r + n * s;
}

__global__ void index_map_kernel(long long* out, int a, int alpha, int w, int gamma, long long n) {
    const long long m = (long long)a * alpha * w;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const int p = int(j % a);
        const int r = int((j / a) % alpha);
        const int s = int(j / ((long long)a * alpha));
        out[j] = stacked_fpa_index(p, r, s, gamma, n);
    }
}

// Calls fn(G{}) for the geometry serving (direction, K, dtype, forward tile
// shape; the adjoint has shape 0 only).
template <class Fn>
int with_geo(bool forward, int K, int dtype, int shape, Fn&& fn) {
    if (shape < 0 || shape >= kFwdShapes || (!forward && shape != 0)) return -1;
    auto by_k = [&](auto tin, auto tf, auto fwd) -> int {
        using TIn = decltype(tin);
        using TF = decltype(tf);
        constexpr bool F = decltype(fwd)::value;
        auto by_shape = [&](auto kc) -> int {
            constexpr int KK = decltype(kc)::value;
            return shape == 1 ? fn(GeoOf<KK, TIn, TF, F, 1>{}) : fn(GeoOf<KK, TIn, TF, F, 0>{});
        };
        switch (K) {
            case 1: return by_shape(std::integral_constant<int, 1>{});
            case 3: return by_shape(std::integral_constant<int, 3>{});
            case 5: return by_shape(std::integral_constant<int, 5>{});
            default: return -1;
        }
    };
    using Fwd = std::integral_constant<bool, true>;
    using Adj = std::integral_constant<bool, false>;
    if (dtype == kDtypeBF16) {
        if (forward) return by_k(__nv_bfloat16{}, __nv_bfloat16{}, Fwd{});
        return by_k(float{}, __nv_bfloat16{}, Adj{});
    }
    if (forward) return by_k(float{}, float{}, Fwd{});
    return by_k(float{}, float{}, Adj{});
}

}  // namespace

// ---------------------------------------------------------------------------
// host entry points used by the plan / API code
// ---------------------------------------------------------------------------
int gather_tile_w(bool forward, int dtype, int shape) {
    return with_geo(forward, 1, dtype, shape, [](auto g) { return decltype(g)::TX; });
}
int gather_tile_h(bool forward, int dtype, int shape) {
    return with_geo(forward, 1, dtype, shape, [](auto g) { return decltype(g)::TY; });
}
int gather_window_rows(bool forward, int K, int dtype, int shape) {
    return gather_tile_h(forward, dtype, shape) + K - 1;
}
int gather_warps_per_cta(bool forward) { return forward ? kShapeFwd.NW : kShapeAdj.NW; }
int gather_box_w(bool forward, int K, int dtype, int shape) {
    return with_geo(forward, K, dtype, shape, [](auto g) { return decltype(g)::BXW; });
}
int gather_weight_pad(bool forward, int K, int dtype) {
    return with_geo(forward, K, dtype, 0, [](auto g) { return decltype(g)::WPAD; });
}
int gather_fwd_shapes() { return kFwdShapes; }
// x-shifted copies of a projector's input: 4 (float32: 16-byte alignment;
// bfloat16: 8-byte alignment, the lanes taking the remaining shift of 0 or 4
// elements inside a 16-byte aligned box)
int gather_input_copies(bool forward, int dtype) {
    (void)forward;
    (void)dtype;
    return 4;
}

cudaError_t gather_prepare(bool forward, int K, int dtype, int* blocks_per_sm, int shape) {
    return forward ? gather_prepare_fwd(K, dtype, shape, blocks_per_sm)
                   : gather_prepare_adj(K, dtype, blocks_per_sm);
}

cudaError_t gather_launch(bool forward, int K, int dtype, const CUtensorMap& win,
                          const GatherParams& p, cudaStream_t stream, int shape) {
    return forward ? gather_launch_fwd(K, dtype, shape, win, p, stream)
                   : gather_launch_adj(K, dtype, win, p, stream);
}

cudaError_t launch_scatter_copies(int dtype, void* dst, long long copy_stride, int ncopies,
                                  int dst_pitch, long long dst_plane_stride, const void* src,
                                  int src_dtype, int src_pitch, long long src_plane_stride,
                                  int width, int height, int planes, float value,
                                  cudaStream_t stream) {
    const int threads = 256, blocks = 2048;
    if (dtype == kDtypeBF16) {
        if (src_dtype == kDtypeBF16)
            scatter_copies_kernel<__nv_bfloat16, __nv_bfloat16><<<blocks, threads, 0, stream>>>(
                static_cast<__nv_bfloat16*>(dst), copy_stride, ncopies, dst_pitch, dst_plane_stride,
                static_cast<const __nv_bfloat16*>(src), src_pitch, src_plane_stride, width, height,
                planes, value);
        else
            scatter_copies_kernel<__nv_bfloat16, float><<<blocks, threads, 0, stream>>>(
                static_cast<__nv_bfloat16*>(dst), copy_stride, ncopies, dst_pitch, dst_plane_stride,
                static_cast<const float*>(src), src_pitch, src_plane_stride, width, height, planes,
                value);
    } else {
        scatter_copies_kernel<float, float><<<blocks, threads, 0, stream>>>(
            static_cast<float*>(dst), copy_stride, ncopies, dst_pitch, dst_plane_stride,
            static_cast<const float*>(src), src_pitch, src_plane_stride, width, height, planes,
            value);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_copy0(int dtype, void* dst, const void* src, int src_pitch,
                                long long src_plane_stride, int width, int height, int planes,
                                cudaStream_t stream) {
    const int threads = 256, blocks = 2048;
    if (dtype == kDtypeBF16)
        gather_copy0_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(
            static_cast<__nv_bfloat16*>(dst), static_cast<const __nv_bfloat16*>(src), src_pitch,
            src_plane_stride, width, height, planes);
    else
        gather_copy0_kernel<float><<<blocks, threads, 0, stream>>>(
            static_cast<float*>(dst), static_cast<const float*>(src), src_pitch, src_plane_stride,
            width, height, planes);
    return cudaGetLastError();
}

#ifdef CTIS_DEBUG_BOUNDS
cudaError_t debug_arm(const void* const lo[6], const size_t bytes[6], unsigned long long* log) {
    DbgRanges r{};
    for (int i = 0; i < 6; ++i) {
        r.lo[i] = static_cast<const char*>(lo[i]);
        r.hi[i] = lo[i] ? static_cast<const char*>(lo[i]) + bytes[i] : nullptr;
    }
    r.log = log;
    cudaError_t e = debug_arm_fwd(r);
    return e != cudaSuccess ? e : debug_arm_adj(r);
}
#endif

cudaError_t launch_frames_gather(float* dst, const float* const* srcs, long long n, int frames,
                                 cudaStream_t stream) {
    frames_gather_kernel<<<2048, 256, 0, stream>>>(dst, srcs, n, frames);
    return cudaGetLastError();
}

cudaError_t launch_frames_scatter_copies(int dtype, void* dst, long long copy_stride, int ncopies,
                                         int dst_pitch, long long dst_plane_stride,
                                         const void* const* srcs, float value, int width,
                                         int height, int planes, int frames, cudaStream_t stream) {
    if (dtype == kDtypeBF16)
        frames_scatter_copies_kernel<__nv_bfloat16><<<2048, 256, 0, stream>>>(
            static_cast<__nv_bfloat16*>(dst), copy_stride, ncopies, dst_pitch, dst_plane_stride,
            reinterpret_cast<const __nv_bfloat16* const*>(srcs), value, width, height, planes,
            frames);
    else
        frames_scatter_copies_kernel<float><<<2048, 256, 0, stream>>>(
            static_cast<float*>(dst), copy_stride, ncopies, dst_pitch, dst_plane_stride,
            reinterpret_cast<const float* const*>(srcs), value, width, height, planes, frames);
    return cudaGetLastError();
}

cudaError_t launch_frames_copy0_out(int dtype, void* const* dsts, const void* src, int src_pitch,
                                    long long src_plane_stride, int width, int height, int planes,
                                    int frames, cudaStream_t stream) {
    if (dtype == kDtypeBF16)
        frames_copy0_out_kernel<__nv_bfloat16><<<2048, 256, 0, stream>>>(
            reinterpret_cast<__nv_bfloat16* const*>(dsts), static_cast<const __nv_bfloat16*>(src),
            src_pitch, src_plane_stride, width, height, planes, frames);
    else
        frames_copy0_out_kernel<float><<<2048, 256, 0, stream>>>(
            reinterpret_cast<float* const*>(dsts), static_cast<const float*>(src), src_pitch,
            src_plane_stride, width, height, planes, frames);
    return cudaGetLastError();
}

cudaError_t launch_rows_scatter(double* dst, const double* src, const int* gid, int len, int frames,
                                cudaStream_t stream) {
    rows_scatter_kernel<<<256, 256, 0, stream>>>(dst, src, gid, len, frames);
    return cudaGetLastError();
}

cudaError_t launch_stats_reduce(double* out, const double* tile_stats, int tiles, int frames,
                                long long frame_stride, double* part, int* tickets,
                                cudaStream_t stream) {
    const int warps_per_block = 4;
    const long long warps = (long long)frames * kStatSlices;
    stats_reduce_kernel<<<int((warps + warps_per_block - 1) / warps_per_block), 32 * warps_per_block,
                          0, stream>>>(out, tile_stats, tiles, frames, frame_stride, part, tickets);
    return cudaGetLastError();
}

cudaError_t launch_index_map(long long* out, int a, int alpha, int w, int gamma, long long n,
                             cudaStream_t stream) {
    index_map_kernel<<<1024, 256, 0, stream>>>(out, a, alpha, w, gamma, n);
    return cudaGetLastError();
}

}  // namespace ctis
