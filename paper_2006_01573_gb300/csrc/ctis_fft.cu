// The paper's own form of the projectors (Sec. 3, Algorithm 1): each block
// H_s = C_s E with C_s the length-n circulant whose first column c_s is the
// calibration image of wavelength s (Eq. 7), so
//     H f   = F^-1 sum_s d_s (.) F v_s,          v_s = E f_s      (Eqs. 11, 13)
//     H^T u = E^T stack_s F^-1 (conj(d_s) (.) F u)                 (Eqs. 14, 17)
// with d_s = F c_s precomputed and F the length-n 1-D real-to-complex Fourier
// transform (Hermitian symmetry: beta = n/2 + 1 coefficients). The transforms
// are cuFFT calls; the index maps, the spectral multiply-accumulate and the EM
// element-wise steps are this file's kernels. Valid when every shifted PSF
// nonzero stays on the FPA (the reject boundary), where the circulant's wrap
// never happens and the form equals the gather projectors.
#include <cufft.h>

#include <cstdint>
#include <new>

#include "ctis_internal.h"
#include "ctis_kernels.h"

namespace ctis {
namespace {

constexpr int kThreads = 256;

int blocks_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads;
    return static_cast<int>(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// v_s = E f_s: datacube element (p, r) of wavelength s to FPA position
// p + gamma * r of the s-th length-n vector (Eq. 11); v is zero elsewhere.
__global__ void embed_kernel(float* v, const float* f, int a, int alpha, int w, int gamma,
                             long long n) {
    const long long m = (long long)a * alpha * w;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const long long ell = (long long)a * alpha;
        const long long s = j / ell, q = j - s * ell;
        const long long p = q % a, r = q / a;
        v[s * n + p + (long long)gamma * r] = f[j];
    }
}

// S = sum_s d_s (.) V_s over the beta coefficients (Eq. 13).
__global__ void mac_kernel(cufftComplex* S, const cufftComplex* D, const cufftComplex* V, int w,
                           long long beta) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < beta;
         k += (long long)gridDim.x * blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int s = 0; s < w; ++s) {
            const cufftComplex d = D[s * beta + k], x = V[s * beta + k];
            re += d.x * x.x - d.y * x.y;
            im += d.x * x.y + d.y * x.x;
        }
        S[k] = make_cuComplex(re, im);
    }
}

// Z_s = conj(d_s) (.) U for every s (Eq. 17).
__global__ void expand_kernel(cufftComplex* Z, const cufftComplex* D, const cufftComplex* U, int w,
                              long long beta) {
    const long long total = beta * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i % beta;
        const cufftComplex d = D[i], u = U[k];
        Z[i] = make_cuComplex(d.x * u.x + d.y * u.y, d.x * u.y - d.y * u.x);
    }
}

// out = in / n (cuFFT's inverse is unnormalised).
__global__ void scale_kernel(float* out, const float* in, long long count, float inv_n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] * inv_n;
}

// zeta = E^T z / n: FPA position p + gamma * r of the s-th vector back to
// datacube element (p, r, s) (the transposed map of Eq. 14).
__global__ void crop_kernel(float* out, const float* z, int a, int alpha, int w, int gamma,
                            long long n, float inv_n) {
    const long long m = (long long)a * alpha * w;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const long long ell = (long long)a * alpha;
        const long long s = j / ell, q = j - s * ell;
        out[j] = z[s * n + q % a + (long long)gamma * (q / a)] * inv_n;
    }
}

// u = g / q with u = 0 where q <= 0 (Eq. 2; q is H f times n, as the inverse
// transform leaves it, so u = n g / q_raw). The transform's rounding leaves
// pixels no footprint meets near, not at, zero: those have g = 0 for any
// measurement H can produce and get u = 0.
__global__ void ratio_kernel(float* u, const float* g, const float* q_raw, long long n, float nf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float q = q_raw[i];
        u[i] = q > 0.f ? nf * g[i] / q : 0.f;
    }
}

// f <- f * (E^T z / n) / h_s, 0 where h_s == 0 (Eq. 2).
__global__ void update_kernel(float* f, const float* z, const float* h, int a, int alpha, int w,
                              int gamma, long long n, float inv_n) {
    const long long m = (long long)a * alpha * w;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const long long ell = (long long)a * alpha;
        const long long s = j / ell, q = j - s * ell;
        const float hs = h[s];
        const float zj = z[s * n + q % a + (long long)gamma * (q / a)] * inv_n;
        f[j] = hs != 0.f ? f[j] * zj / hs : 0.f;
    }
}

__global__ void fill_kernel(float* out, long long count, float value) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = value;
}

}  // namespace

struct FftForm {
    int a = 0, alpha = 0, w = 0, gamma = 0, xi = 0;
    long long n = 0, beta = 0;
    cufftHandle r2c_w = 0, c2r_w = 0, r2c_1 = 0, c2r_1 = 0;
    bool have_r2c_w = false, have_c2r_w = false, have_r2c_1 = false, have_c2r_1 = false;
    cufftComplex* D = nullptr;   // [w][beta] d_s = F c_s
    cufftComplex* X = nullptr;   // [w][beta] spectra of the w vectors
    cufftComplex* S = nullptr;   // [beta]
    float* v = nullptr;          // [w][n] v_s = E f_s: zero off the embedded positions
    float* z = nullptr;          // [w][n] the adjoint's inverse transforms
    float* q = nullptr;          // [n]
    float* hd = nullptr;         // [w] h per wavelength
};

namespace {

cudaError_t cufft_err(cufftResult r) {
    return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace

void fft_form_destroy(FftForm* F) {
    if (!F) return;
    if (F->have_r2c_w) cufftDestroy(F->r2c_w);
    if (F->have_c2r_w) cufftDestroy(F->c2r_w);
    if (F->have_r2c_1) cufftDestroy(F->r2c_1);
    if (F->have_c2r_1) cufftDestroy(F->c2r_1);
    cudaFree(F->D);
    cudaFree(F->X);
    cudaFree(F->S);
    cudaFree(F->v);
    cudaFree(F->z);
    cudaFree(F->q);
    cudaFree(F->hd);
    delete F;
}

cudaError_t fft_form_create(FftForm** out, int a, int alpha, int w, int gamma, int xi,
                            const float* calib_host, const float* h_host) {
    *out = nullptr;
    FftForm* F = new (std::nothrow) FftForm();
    if (!F) return cudaErrorMemoryAllocation;
    F->a = a;
    F->alpha = alpha;
    F->w = w;
    F->gamma = gamma;
    F->xi = xi;
    F->n = (long long)gamma * xi;
    F->beta = F->n / 2 + 1;
    const long long n = F->n, beta = F->beta;
    cudaError_t e = cudaMalloc(&F->D, sizeof(cufftComplex) * beta * w);
    if (e == cudaSuccess) e = cudaMalloc(&F->X, sizeof(cufftComplex) * beta * w);
    if (e == cudaSuccess) e = cudaMalloc(&F->S, sizeof(cufftComplex) * beta);
    if (e == cudaSuccess) e = cudaMalloc(&F->v, sizeof(float) * n * w);
    if (e == cudaSuccess) e = cudaMalloc(&F->z, sizeof(float) * n * w);
    if (e == cudaSuccess) e = cudaMalloc(&F->q, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&F->hd, sizeof(float) * w);
    int nn = static_cast<int>(n);
    if (e == cudaSuccess)
        e = cufft_err(cufftPlanMany(&F->r2c_w, 1, &nn, nullptr, 1, nn, nullptr, 1,
                                    static_cast<int>(beta), CUFFT_R2C, w));
    F->have_r2c_w = e == cudaSuccess;
    if (e == cudaSuccess)
        e = cufft_err(cufftPlanMany(&F->c2r_w, 1, &nn, nullptr, 1, static_cast<int>(beta), nullptr,
                                    1, nn, CUFFT_C2R, w));
    F->have_c2r_w = e == cudaSuccess;
    if (e == cudaSuccess) e = cufft_err(cufftPlan1d(&F->r2c_1, nn, CUFFT_R2C, 1));
    F->have_r2c_1 = e == cudaSuccess;
    if (e == cudaSuccess) e = cufft_err(cufftPlan1d(&F->c2r_1, nn, CUFFT_C2R, 1));
    F->have_c2r_1 = e == cudaSuccess;
    // d_s = F c_s, once (Eq. 13)
    if (e == cudaSuccess)
        e = cudaMemcpy(F->v, calib_host, sizeof(float) * n * w, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(F->hd, h_host, sizeof(float) * w, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cufft_err(cufftExecR2C(F->r2c_w, F->v, F->D));
    // v then holds only E f_s: the embedding rewrites the same positions
    // every time and nothing else writes v (an out-of-place real-to-complex
    // transform leaves its input as it was)
    if (e == cudaSuccess) e = cudaMemset(F->v, 0, sizeof(float) * n * w);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fft_form_destroy(F);
        return e;
    }
    *out = F;
    return cudaSuccess;
}

// raw = n * H f (no 1/n yet), into F->q.
static cudaError_t forward_raw(FftForm* F, const float* f, cudaStream_t st) {
    const long long n = F->n, beta = F->beta, m = (long long)F->a * F->alpha * F->w;
    cudaError_t e;
    embed_kernel<<<blocks_for(m), kThreads, 0, st>>>(F->v, f, F->a, F->alpha, F->w, F->gamma, n);
    e = cufft_err(cufftSetStream(F->r2c_w, st));
    if (e == cudaSuccess) e = cufft_err(cufftExecR2C(F->r2c_w, F->v, F->X));
    if (e != cudaSuccess) return e;
    mac_kernel<<<blocks_for(beta), kThreads, 0, st>>>(F->S, F->D, F->X, F->w, beta);
    e = cufft_err(cufftSetStream(F->c2r_1, st));
    if (e == cudaSuccess) e = cufft_err(cufftExecC2R(F->c2r_1, F->S, F->q));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// F->z = n * stack_s C_s^T u (no 1/n yet).
static cudaError_t adjoint_raw(FftForm* F, const float* u, cudaStream_t st) {
    const long long beta = F->beta;
    cudaError_t e = cufft_err(cufftSetStream(F->r2c_1, st));
    if (e == cudaSuccess) e = cufft_err(cufftExecR2C(F->r2c_1, const_cast<float*>(u), F->S));
    if (e != cudaSuccess) return e;
    expand_kernel<<<blocks_for(beta * F->w), kThreads, 0, st>>>(F->X, F->D, F->S, F->w, beta);
    e = cufft_err(cufftSetStream(F->c2r_w, st));
    if (e == cudaSuccess) e = cufft_err(cufftExecC2R(F->c2r_w, F->X, F->z));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t fft_form_forward(FftForm* F, const float* f, float* hf, cudaStream_t st) {
    cudaError_t e = forward_raw(F, f, st);
    if (e != cudaSuccess) return e;
    scale_kernel<<<blocks_for(F->n), kThreads, 0, st>>>(hf, F->q, F->n, 1.0f / float(F->n));
    return cudaGetLastError();
}

cudaError_t fft_form_adjoint(FftForm* F, const float* u, float* out, cudaStream_t st) {
    cudaError_t e = adjoint_raw(F, u, st);
    if (e != cudaSuccess) return e;
    const long long m = (long long)F->a * F->alpha * F->w;
    crop_kernel<<<blocks_for(m), kThreads, 0, st>>>(out, F->z, F->a, F->alpha, F->w, F->gamma, F->n,
                                                    1.0f / float(F->n));
    return cudaGetLastError();
}

// k EM updates (Algorithm 1) from f (read) or ones (init_ones), in place.
// u_work: n floats of workspace.
cudaError_t fft_form_reconstruct(FftForm* F, const float* g, float* f, float* u_work, int k,
                                 bool init_ones, cudaStream_t st) {
    const long long m = (long long)F->a * F->alpha * F->w;
    if (init_ones) fill_kernel<<<blocks_for(m), kThreads, 0, st>>>(f, m, 1.0f);
    for (int it = 0; it < k; ++it) {
        cudaError_t e = forward_raw(F, f, st);
        if (e != cudaSuccess) return e;
        ratio_kernel<<<blocks_for(F->n), kThreads, 0, st>>>(u_work, g, F->q, F->n, float(F->n));
        e = adjoint_raw(F, u_work, st);
        if (e != cudaSuccess) return e;
        update_kernel<<<blocks_for(m), kThreads, 0, st>>>(f, F->z, F->hd, F->a, F->alpha, F->w,
                                                          F->gamma, F->n, 1.0f / float(F->n));
    }
    return cudaGetLastError();
}

}  // namespace ctis
