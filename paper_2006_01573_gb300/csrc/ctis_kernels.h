// Host-side launch interface of the CUDA kernels (C++ linkage, library-internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "ctis_internal.h"

namespace ctis {

constexpr int kDtypeF32 = 0;
constexpr int kDtypeBF16 = 1;

// Geometry of the instantiations serving each direction (forward = true) and,
// for the forward, tile shape (0: 32 x 32 tiles, 1: 32 x 16; the adjoint has
// shape 0 only). Invalid combinations return -1.
int gather_tile_w(bool forward, int dtype, int shape = 0);   // output tile columns
int gather_tile_h(bool forward, int dtype, int shape = 0);   // output tile rows
int gather_window_rows(bool forward, int K, int dtype, int shape = 0);   // TMA box height
int gather_warps_per_cta(bool forward);
int gather_box_w(bool forward, int K, int dtype, int shape = 0);   // TMA box width (elements)
int gather_weight_pad(bool forward, int K, int dtype);  // weight words per cluster, padded
int gather_input_copies(bool forward, int dtype);       // x-shifted copies of the input
int gather_fwd_shapes();                                // forward tile shapes built

// Sets kernel attributes and returns the number of resident CTAs per SM for
// the instantiation serving (direction, K, dtype, shape). Call before capture.
cudaError_t gather_prepare(bool forward, int K, int dtype, int* blocks_per_sm, int shape = 0);

// Enqueues one projector pass over p.n_warps independent warps. `win` is the
// tensor map of the input copies with box (box_w, window_rows, 1).
cudaError_t gather_launch(bool forward, int K, int dtype, const CUtensorMap& win,
                          const GatherParams& p, cudaStream_t stream, int shape = 0);

// The ratio step of a wavelength-sharded EM iteration (ctis_shard.cu): u = g
// / q (0 where q = 0) into the FPA copies; with stats_out, the four
// statistics of (q, g) over q > 0 into stats_out[0..3] through `part`
// ([shard_ratio_blocks()][kNumStats] float64 scratch), in a fixed order.
int shard_ratio_blocks();
cudaError_t launch_shard_ratio(float* copies, long long copy_stride, int ncopies, int pitch,
                               const float* q, const float* g, int width, int height, double* part,
                               double* stats_out, cudaStream_t stream);

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

// Frame totals of a forward's tile statistics (kStatSlices warps per frame,
// fixed order): out + f * frame_stride <- sum over tile_stats[f][0..tiles).
// part: [frames][kStatSlices][kNumStats] scratch; tickets: [frames], zero
// before and after.
cudaError_t launch_stats_reduce(double* out, const double* tile_stats, int tiles, int frames,
                                long long frame_stride, double* part, int* tickets,
                                cudaStream_t stream);

// ---- frames of a batch (srcs / dsts: device arrays of per-frame pointers)
// dst[f * n + i] = srcs[f][i]
cudaError_t launch_frames_gather(float* dst, const float* const* srcs, long long n, int frames,
                                 cudaStream_t stream);
// x-shifted copies of the frames' datacubes (frame f, plane z -> copies'
// plane f * planes + z), from srcs (plan dtype) or the constant `value`
cudaError_t launch_frames_scatter_copies(int dtype, void* dst, long long copy_stride, int ncopies,
                                         int dst_pitch, long long dst_plane_stride,
                                         const void* const* srcs, float value, int width,
                                         int height, int planes, int frames, cudaStream_t stream);
// copy 0 of the frames' datacubes back to dense per-frame buffers
cudaError_t launch_frames_copy0_out(int dtype, void* const* dsts, const void* src, int src_pitch,
                                    long long src_plane_stride, int width, int height, int planes,
                                    int frames, cudaStream_t stream);
// dst row gid[f] <- src row f (rows of len doubles)
cudaError_t launch_rows_scatter(double* dst, const double* src, const int* gid, int len, int frames,
                                cudaStream_t stream);

// ---- gradients (ctis_gather_grad.cu)
// PSF-value gradient pass over the adjoint's work lists (mode kEpiGrad).
cudaError_t psf_grad_prepare(int K, int dtype, int* blocks_per_sm);
cudaError_t psf_grad_launch(int K, int dtype, const CUtensorMap& win, const GatherParams& p,
                            cudaStream_t stream);
// dval[t] (+)= sum over the plane's tiles of the partial sums of tap t, plus
// extra[tap_s[t]] when extra is not null.
cudaError_t launch_grad_reduce(float* dval, const float* part, const int* slot, const int* tap_s,
                               const double* extra, int nnz, int kk, int tiles_per_plane,
                               bool accumulate, cudaStream_t stream);
// FPA values into the adjoint's x-shifted copies: mode 0 u = g / q, mode 1
// gq = -gu * g / q^2 (0 where q == 0).
cudaError_t launch_fpa_to_copies(float* copies, long long copy_stride, int ncopies, int pitch,
                                 const float* q, const float* g, const float* gu, int width,
                                 int height, int mode, cudaStream_t stream);
// Vector-Jacobian product of f' = f * z / h_s: a = gb f / h_s (dense and into
// the datacube copies), gfd = gb z / h_s, per-plane float64 partials of
// gb f z; launch_dh_finish turns them into dL/dh_s. With h_vox (h per voxel)
// h_j replaces h_s and dL/dh_j goes to dh_vox per voxel.
int voxel_vjp_blocks();
cudaError_t launch_voxel_vjp(float* a_dense, float* a_copies, long long copy_stride, int ncopies,
                             int pitch, long long plane_stride, float* gfd, double* part,
                             const float* gb, const float* f, const float* z, const float* h,
                             int a, int alpha, int w, const float* h_vox, float* dh_vox,
                             cudaStream_t stream);
cudaError_t launch_dh_finish(double* dh, const double* part, const float* h, int w,
                             cudaStream_t stream);
cudaError_t launch_add(float* out, const float* x, const float* y, long long n,
                       cudaStream_t stream);
cudaError_t launch_negate(double* out, const double* in, cudaStream_t stream);

// The paper's FFT form of the projectors (ctis_fft.cu): H_s = C_s E with
// circulant C_s (Eqs. 7, 11, 13, 14, 17), the transforms by cuFFT.
// calib_host: [w][n] float32 calibration images c_s; h_host: [w].
struct FftForm;
cudaError_t fft_form_create(FftForm** out, int a, int alpha, int w, int gamma, int xi,
                            const float* calib_host, const float* h_host);
void fft_form_destroy(FftForm* F);
cudaError_t fft_form_forward(FftForm* F, const float* f, float* hf, cudaStream_t st);
cudaError_t fft_form_adjoint(FftForm* F, const float* u, float* out, cudaStream_t st);
cudaError_t fft_form_reconstruct(FftForm* F, const float* g, float* f, float* u_work, int k,
                                 bool init_ones, cudaStream_t st);

}  // namespace ctis
