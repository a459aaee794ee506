// Host-side launch interface of the CUDA kernels (C++ linkage, library-internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "ctis_internal.h"

namespace ctis {

constexpr int kDtypeF32 = 0;
constexpr int kDtypeBF16 = 1;

// Output tile of one work item and the TMA box of one input window.
int gather_tile_w();
int gather_tile_h();
int gather_window_rows(int K);        // LY*R + K - 1 rows
int gather_box_w(int K, int dtype);     // TMA box width of the forward's f windows
int gather_box_w_input_f32(int K);      // TMA box width of the adjoint's FPA windows

// Sets kernel attributes and returns the number of resident CTAs per SM for
// the instantiation serving (direction, K, dtype). Call before capture.
cudaError_t gather_prepare(bool forward, int K, int dtype, int* blocks_per_sm);

// Enqueues one projector pass over p.n_warps independent warps. `slab` is the
// tensor map of the input planes with box (box_w, R, 1); `halo` the same map
// with box (box_w, K - 1, 1).
cudaError_t gather_launch(bool forward, int K, int dtype, const CUtensorMap& slab,
                          const CUtensorMap& halo, const GatherParams& p, cudaStream_t stream);
int gather_warps_per_cta();

cudaError_t launch_fill(int dtype, void* f, int a, int rows, int pitch, float value,
                        cudaStream_t stream);
cudaError_t launch_index_map(long long* out, int a, int alpha, int w, int gamma, long long n,
                             cudaStream_t stream);

}  // namespace ctis
