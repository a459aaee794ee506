// Host-side launch interface of the CUDA kernels (C++ linkage, library-internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "ctis_internal.h"

namespace ctis {

constexpr int kDtypeF32 = 0;
constexpr int kDtypeBF16 = 1;

// Geometry of the instantiations serving each direction (forward = true).
int gather_tile_w(bool forward, int dtype);         // output tile columns
int gather_tile_h(bool forward, int dtype);         // output tile rows
int gather_window_rows(bool forward, int K, int dtype);   // TMA box height (tile rows + K - 1)
int gather_warps_per_cta(bool forward);
int gather_box_w(bool forward, int K, int dtype);   // TMA box width (elements)
int gather_weight_pad(bool forward, int K, int dtype);  // weight pairs per cluster, padded
int gather_input_copies(bool forward, int dtype);       // x-shifted copies of the input

// Sets kernel attributes and returns the number of resident CTAs per SM for
// the instantiation serving (direction, K, dtype). Call before capture.
cudaError_t gather_prepare(bool forward, int K, int dtype, int* blocks_per_sm);

// Enqueues one projector pass over p.n_warps independent warps. `win` is the
// tensor map of the input copies with box (box_w, window_rows, 1).
cudaError_t gather_launch(bool forward, int K, int dtype, const CUtensorMap& win,
                          const GatherParams& p, cudaStream_t stream);

// Writes the x-shifted copies (copy q, element x + q = src[x]) of a plane
// stack from `src` (any pitch; src_dtype float32 or the copies' dtype), or of
// the constant `value` when src is null.
cudaError_t launch_scatter_copies(int dtype, void* dst, long long copy_stride, int ncopies,
                                  int dst_pitch, long long dst_plane_stride, const void* src,
                                  int src_dtype, int src_pitch, long long src_plane_stride,
                                  int width, int height, int planes, float value,
                                  cudaStream_t stream);
// Copies copy 0 of a plane stack into a dense buffer.
cudaError_t launch_gather_copy0(int dtype, void* dst, const void* src, int src_pitch,
                                long long src_plane_stride, int width, int height, int planes,
                                cudaStream_t stream);
#ifdef CTIS_DEBUG_BOUNDS
// Registers the buffers epilogue accesses may touch (debug builds only).
cudaError_t debug_arm(const void* const lo[6], const size_t bytes[6], unsigned long long* log);
#endif
// Fixed scratch array of ctis_forward_static_scratch (ctis_static_scratch.cu).
size_t static_scratch_bytes();
cudaError_t static_scratch_ptr(void** out);   // device address on the current device

cudaError_t launch_index_map(long long* out, int a, int alpha, int w, int gamma, long long n,
                             cudaStream_t stream);

}  // namespace ctis
