/*
 * C caller of libslab.so through include/slab.h only (no Python, no ctypes zero-filling).
 *
 * Usage: abi_check n b kappa.bin f.bin out.bin
 *   kappa.bin: (n+1)^2 doubles, f.bin: (n-1)^2 doubles (one load, also used as dL/du).
 * Factors the 2-D diffusion problem twice -- once with opts == NULL, once with a slab_opts
 * struct whose bytes were set to 0xFF before slab_default_opts filled it -- and writes
 *   int32 status[6]  (factor NULL, solve, adjoint, factor defaults, solve, destroy-ok = 0)
 *   double relres[2], u_null[N], lambda[N], grad[(n+1)^2], u_defaults[N]
 * to out.bin.  Exit code 0 when every call returned SLAB_OK.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "slab.h"

static int read_all(const char* path, double* dst, size_t count) {
    FILE* fp = fopen(path, "rb");
    if (!fp) return 0;
    const size_t got = fread(dst, sizeof(double), count, fp);
    fclose(fp);
    return got == count;
}

static void* dev_alloc(size_t bytes) {
    void* p = NULL;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc(%zu) failed\n", bytes);
        exit(3);
    }
    return p;
}

int main(int argc, char** argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s n b kappa.bin f.bin out.bin\n", argv[0]);
        return 2;
    }
    const int n = atoi(argv[1]), b = atoi(argv[2]);
    const size_t N = (size_t)(n - 1) * (n - 1), NN = (size_t)(n + 1) * (n + 1);
    double* kappa = (double*)malloc(NN * sizeof(double));
    double* f = (double*)malloc(N * sizeof(double));
    double* out = (double*)malloc((3 * N + NN) * sizeof(double));
    if (!kappa || !f || !out || !read_all(argv[3], kappa, NN) || !read_all(argv[4], f, N)) {
        fprintf(stderr, "cannot read inputs\n");
        return 2;
    }
    double *dk = (double*)dev_alloc(NN * 8), *df = (double*)dev_alloc(N * 8), *du = (double*)dev_alloc(N * 8);
    double *dl = (double*)dev_alloc(N * 8), *dg = (double*)dev_alloc(NN * 8), *du2 = (double*)dev_alloc(N * 8);
    cudaMemcpy(dk, kappa, NN * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(df, f, N * 8, cudaMemcpyHostToDevice);
    cudaMemset(dg, 0, NN * 8);

    slab_grid grid = {2, n};
    slab_coeffs co = {SLAB_DIFFUSION, dk, NULL, 0.0};
    int status[6] = {-1, -1, -1, -1, -1, 0};
    double relres[2] = {-1.0, -1.0};
    int iters = -1;

    /* 1. opts == NULL: the library's defaults */
    slab_handle* h = NULL;
    status[0] = slab_factor(&grid, &co, b, NULL, &h);
    if (status[0] == SLAB_OK) {
        status[1] = slab_solve(h, df, du, 1, &relres[0], &iters);
        status[2] = slab_adjoint(h, df, du, dl, dg, 1);
        slab_destroy(h);
    }

    /* 2. a struct full of 0xFF bytes, then slab_default_opts: every field must be set */
    slab_opts o;
    memset(&o, 0xFF, sizeof(o));
    slab_default_opts(&o);
    h = NULL;
    status[3] = slab_factor(&grid, &co, b, &o, &h);
    if (status[3] == SLAB_OK) {
        status[4] = slab_solve(h, df, du2, 1, &relres[1], &iters);
        slab_destroy(h);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) status[5] = SLAB_ECUDA;

    cudaMemcpy(out, du, N * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out + N, dl, N * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out + 2 * N, dg, NN * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out + 2 * N + NN, du2, N * 8, cudaMemcpyDeviceToHost);
    FILE* fp = fopen(argv[5], "wb");
    if (!fp) return 2;
    fwrite(status, sizeof(int), 6, fp);
    fwrite(relres, sizeof(double), 2, fp);
    fwrite(out, sizeof(double), 3 * N + NN, fp);
    fclose(fp);
    for (int i = 0; i < 6; ++i)
        if (status[i] != SLAB_OK) {
            fprintf(stderr, "call %d returned %d (%s)\n", i, status[i], slab_strerror((slab_status)status[i]));
            return 1;
        }
    printf("abi_check ok: relres %.2e %.2e\n", relres[0], relres[1]);
    return 0;
}
