// Gradients with respect to the PSF values, and the element-wise steps of the
// unrolled EM gradient.
//
// The PSF-value gradient of <r, H f> is, for every stored tap t of
// wavelength s at FPA offset (x_t, y_t),
//     dval_t = sum_{p,r} f_s(p, r) * r(x_t + p, y_t + r),
// because tap t adds v_t f_s(p, r) to pixel (x_t + p, y_t + r) (Sec. 2
// shift-invariance). It reads exactly what the adjoint reads: for a voxel
// tile of wavelength s and a spot cluster of s, the FPA window at the
// cluster's offset. The kernel therefore runs the adjoint's work lists and
// TMA pipeline; per task, every lane multiplies its block of f_s with the
// window at the K x K offsets, the warp adds the lanes' sums, and the task
// writes its K x K partial sums. A second kernel adds the partials of every
// tap over the voxel tiles of its plane in a fixed order.
#include "ctis_gather.cuh"

namespace ctis {
namespace {

template <class G, typename TIn, typename TF, int MODE>
__global__ void __launch_bounds__(G::THREADS, G::MIN_BLOCKS)
    psf_grad_kernel(const __grid_constant__ CUtensorMap tm_win, const GatherParams p) {
    gather_body<G, TIn, TF, MODE>(tm_win, p);
}

template <class Fn>
cudaError_t dispatch_grad(int K, int dtype, Fn&& fn) {
    auto by_k = [&](auto tin, auto tf) -> cudaError_t {
        using TIn = decltype(tin);
        using TF = decltype(tf);
        switch (K) {
            case 1: return fn(psf_grad_kernel<GeoOf<1, TIn, TF, false>, TIn, TF, kEpiGrad>,
                              GeoOf<1, TIn, TF, false>{});
            case 3: return fn(psf_grad_kernel<GeoOf<3, TIn, TF, false>, TIn, TF, kEpiGrad>,
                              GeoOf<3, TIn, TF, false>{});
            case 5: return fn(psf_grad_kernel<GeoOf<5, TIn, TF, false>, TIn, TF, kEpiGrad>,
                              GeoOf<5, TIn, TF, false>{});
            default: return cudaErrorInvalidValue;
        }
    };
    if (dtype == kDtypeBF16) return by_k(float{}, __nv_bfloat16{});
    return by_k(float{}, float{});
}

// dval[t] (+)= sum over the plane's voxel tiles of the partial sums of tap t's
// cluster slot, plus extra[s_t] when given. slot[t] = cluster * K*K + dy*K + dx.
__global__ void grad_reduce_kernel(float* dval, const float* part, const int* slot,
                                   const int* tap_s, const double* extra, int nnz, int kk,
                                   int tiles_per_plane, int accumulate) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += gridDim.x * blockDim.x) {
        const int sl = slot[t];
        const int c = sl / kk, e = sl - c * kk;
        const float* src = part + (long long)c * tiles_per_plane * kk + e;
        float sum = 0.f;
        for (int i = 0; i < tiles_per_plane; ++i) sum += src[(long long)i * kk];
        double d = sum;
        if (extra) d += extra[tap_s[t]];
        dval[t] = accumulate ? float(double(dval[t]) + d) : float(d);
    }
}

// Element-wise FPA steps written straight into the x-shifted copies of the
// adjoint's input (copy q, element x + q):
//   mode 0: u  = g / q                       (Eq. 2 ratio; 0 where q == 0)
//   mode 1: gq = -gu * g / q^2               (derivative of u = g / q)
__global__ void fpa_to_copies_kernel(float* copies, long long copy_stride, int ncopies, int pitch,
                                     const float* q, const float* g, const float* gu, int width,
                                     int height, int mode) {
    const long long n = (long long)width * height;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % width);
        const long long y = i / width;
        const float qv = q[i];
        float v = 0.f;
        if (qv > 0.f) v = mode == 0 ? g[i] / qv : -gu[i] * g[i] / (qv * qv);
        float* d = copies + y * pitch + x;
        for (int c = 0; c < ncopies; ++c) d[c * copy_stride + c] = v;
    }
}

// Element-wise datacube step of the EM update's vector-Jacobian product, for
// f' = f * z / h_s with incoming gradient gb = dL/df':
//   a   = gb * f / h_s     (gradient reaching z), scattered into the copies;
//   gfd = gb * z / h_s     (direct part of dL/df);
//   part[s][block] = sum over the block of gb * f * z  (float64), from which
//   dL/dh_s = -sum / h_s^2.
// With h per voxel (h_vox, the clipped boundary) the same with h_j in place
// of h_s, and dL/dh_j = -gb f z / h_j^2 per voxel into dh_vox (0 where
// h_j == 0).
// Grid: (blocks per plane, w); each block sums its slice in a fixed order.
constexpr int kVjpThreads = 256;
__global__ void __launch_bounds__(kVjpThreads)
    voxel_vjp_kernel(float* a_dense, float* a_copies, long long copy_stride, int ncopies,
                     int pitch, long long plane_stride, float* gfd, double* part,
                     const float* gb, const float* f, const float* z, const float* h, int a,
                     int alpha, const float* h_vox, float* dh_vox) {
    const int s = blockIdx.y;
    const long long plane = (long long)a * alpha;
    const float hs = h[s];
    const float rh_s = hs != 0.f ? 1.0f / hs : 0.f;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = s * plane + i;
        const float gv = gb[j], fv = f[j], zv = z[j];
        float rh = rh_s;
        if (h_vox) {
            const float hj = h_vox[j];
            rh = hj != 0.f ? 1.0f / hj : 0.f;
            dh_vox[j] = -gv * fv * zv * rh * rh;
        }
        const float av = gv * fv * rh;
        a_dense[j] = av;
        gfd[j] = gv * zv * rh;
        acc += double(gv) * double(fv) * double(zv);
        const int x = int(i % a);
        const long long y = i / a;
        float* d = a_copies + s * plane_stride + y * pitch + x;
        for (int c = 0; c < ncopies; ++c) d[c * copy_stride + c] = av;
    }
    __shared__ double red[kVjpThreads / 32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kVjpThreads / 32; ++k) t += red[k];
        part[(long long)s * gridDim.x + blockIdx.x] = t;
    }
}

// dL/dh_s = -(sum of the plane's partials, in block order) / h_s^2 (0 where
// h_s == 0, where the update sets f = 0 whatever h is).
__global__ void dh_finish_kernel(double* dh, const double* part, int blocks, const float* h, int w) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= w) return;
    double t = 0.0;
    for (int b = 0; b < blocks; ++b) t += part[(long long)s * blocks + b];
    const double hs = h[s];
    dh[s] = hs != 0.0 ? -t / (hs * hs) : 0.0;
}

__global__ void negate_kernel(double* out, const double* in) { out[0] = -in[0]; }

__global__ void add_kernel(float* out, const float* x, const float* y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = x[i] + y[i];
}

}  // namespace

cudaError_t psf_grad_prepare(int K, int dtype, int* blocks_per_sm) {
    return dispatch_grad(K, dtype, [&](auto kern, auto geo) {
        return prepare_kernel<decltype(geo)>(kern, blocks_per_sm);
    });
}

cudaError_t psf_grad_launch(int K, int dtype, const CUtensorMap& win, const GatherParams& p,
                            cudaStream_t stream) {
    return dispatch_grad(K, dtype, [&](auto kern, auto geo) {
        return launch_kernel<decltype(geo)>(kern, win, p, stream);
    });
}

cudaError_t launch_grad_reduce(float* dval, const float* part, const int* slot, const int* tap_s,
                               const double* extra, int nnz, int kk, int tiles_per_plane,
                               bool accumulate, cudaStream_t stream) {
    const int threads = 256, blocks = (nnz + threads - 1) / threads;
    if (blocks == 0) return cudaSuccess;
    grad_reduce_kernel<<<blocks, threads, 0, stream>>>(dval, part, slot, tap_s, extra, nnz, kk,
                                                       tiles_per_plane, accumulate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_fpa_to_copies(float* copies, long long copy_stride, int ncopies, int pitch,
                                 const float* q, const float* g, const float* gu, int width,
                                 int height, int mode, cudaStream_t stream) {
    fpa_to_copies_kernel<<<1024, 256, 0, stream>>>(copies, copy_stride, ncopies, pitch, q, g, gu,
                                                   width, height, mode);
    return cudaGetLastError();
}

int voxel_vjp_blocks() { return 32; }

cudaError_t launch_voxel_vjp(float* a_dense, float* a_copies, long long copy_stride, int ncopies,
                             int pitch, long long plane_stride, float* gfd, double* part,
                             const float* gb, const float* f, const float* z, const float* h,
                             int a, int alpha, int w, const float* h_vox, float* dh_vox,
                             cudaStream_t stream) {
    dim3 grid(voxel_vjp_blocks(), w);
    voxel_vjp_kernel<<<grid, kVjpThreads, 0, stream>>>(a_dense, a_copies, copy_stride, ncopies,
                                                       pitch, plane_stride, gfd, part, gb, f, z,
                                                       h, a, alpha, h_vox, dh_vox);
    return cudaGetLastError();
}

cudaError_t launch_dh_finish(double* dh, const double* part, const float* h, int w,
                             cudaStream_t stream) {
    dh_finish_kernel<<<(w + 127) / 128, 128, 0, stream>>>(dh, part, voxel_vjp_blocks(), h, w);
    return cudaGetLastError();
}

cudaError_t launch_add(float* out, const float* x, const float* y, long long n,
                       cudaStream_t stream) {
    add_kernel<<<1024, 256, 0, stream>>>(out, x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_negate(double* out, const double* in, cudaStream_t stream) {
    negate_kernel<<<1, 1, 0, stream>>>(out, in);
    return cudaGetLastError();
}

}  // namespace ctis
