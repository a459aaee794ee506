/* A plain C99 caller of the C ABI on the GPU, with no Python or PyTorch:
 * reads a problem from stdin (sizes, the PSF, the FPA image), creates a plan,
 * runs k EM updates with statistics through ctis_reconstruct, and prints the
 * reconstruction and the statistics. Device memory comes from the CUDA
 * runtime. Compiled and run by tests/test_gpu_14_c_caller.py, which checks
 * the output against the FP64 oracle.
 *
 * stdin:  a alpha w gamma xi k
 *         nnz, then psf_ptr[w + 1], then nnz lines "x y v"
 *         gamma * xi values of g (row-major)
 * stdout: m values of f, then (k + 1) * 4 statistics */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "ctis.h"

static int check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
        return 1;
    }
    return 0;
}

int main(void) {
    int a, alpha, w, gamma, xi, k, nnz;
    if (scanf("%d %d %d %d %d %d %d", &a, &alpha, &w, &gamma, &xi, &k, &nnz) != 7) return 2;
    int32_t* ptr = malloc(sizeof(int32_t) * (size_t)(w + 1));
    int32_t* x = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t* y = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    float* v = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    const size_t m = (size_t)a * alpha * w, n = (size_t)gamma * xi;
    float* g = malloc(sizeof(float) * n);
    float* f = malloc(sizeof(float) * m);
    double* st = malloc(sizeof(double) * (size_t)(k + 1) * CTIS_NSTATS);
    if (!ptr || !x || !y || !v || !g || !f || !st) return 3;
    for (int s = 0; s <= w; ++s)
        if (scanf("%d", &ptr[s]) != 1) return 2;
    for (int i = 0; i < nnz; ++i)
        if (scanf("%d %d %f", &x[i], &y[i], &v[i]) != 3) return 2;
    for (size_t i = 0; i < n; ++i)
        if (scanf("%f", &g[i]) != 1) return 2;

    ctis_plan* plan = NULL;
    int rc = ctis_plan_create(&plan, a, alpha, w, gamma, xi, ptr, x, y, v, CTIS_F32);
    if (rc != CTIS_OK) {
        fprintf(stderr, "plan: %s (%s)\n", ctis_status_string(rc), ctis_last_error());
        return 1;
    }
    float *g_dev = NULL, *f_dev = NULL;
    double* st_dev = NULL;
    if (check_cuda(cudaMalloc((void**)&g_dev, sizeof(float) * n), "cudaMalloc g") ||
        check_cuda(cudaMalloc((void**)&f_dev, sizeof(float) * m), "cudaMalloc f") ||
        check_cuda(cudaMalloc((void**)&st_dev, sizeof(double) * (size_t)(k + 1) * CTIS_NSTATS),
                   "cudaMalloc stats") ||
        check_cuda(cudaMemcpy(g_dev, g, sizeof(float) * n, cudaMemcpyHostToDevice), "copy g"))
        return 1;
    rc = ctis_reconstruct(plan, g_dev, f_dev, k, CTIS_INIT_ONES, st_dev, NULL);
    if (rc == CTIS_OK) rc = ctis_plan_check(plan, NULL);
    if (rc != CTIS_OK) {
        fprintf(stderr, "reconstruct: %s (%s)\n", ctis_status_string(rc), ctis_last_error());
        return 1;
    }
    if (check_cuda(cudaMemcpy(f, f_dev, sizeof(float) * m, cudaMemcpyDeviceToHost), "copy f") ||
        check_cuda(cudaMemcpy(st, st_dev, sizeof(double) * (size_t)(k + 1) * CTIS_NSTATS,
                              cudaMemcpyDeviceToHost), "copy stats"))
        return 1;
    for (size_t j = 0; j < m; ++j) printf("%.9g\n", f[j]);
    for (int i = 0; i < (k + 1) * CTIS_NSTATS; ++i) printf("%.17g\n", st[i]);
    ctis_plan_destroy(plan);
    cudaFree(g_dev);
    cudaFree(f_dev);
    cudaFree(st_dev);
    free(ptr); free(x); free(y); free(v); free(g); free(f); free(st);
    return 0;
}
