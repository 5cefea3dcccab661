/*
 * Calls libgfc through its C ABI alone (no Python, no PyTorch): evaluates
 * the D = 4 bubble on a small cell-centred grid (Kernel 1 fused into Kernel 2,
 * Sect. 4 of the paper) in FP64 and prints "i j re im" per point, then one
 * line of counters. Built and run by tests/test_c_abi_gpu.py.
 *
 * usage: c_abi_example M N n_radial n_angular
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "gfc.h"

int main(int argc, char **argv)
{
    if (argc != 5) {
        fprintf(stderr, "usage: %s M N n_radial n_angular\n", argv[0]);
        return 2;
    }
    int m = atoi(argv[1]), n = atoi(argv[2]);
    gfc_propagator prop = {0};
    prop.kind = GFC_PROP_SCALAR;
    prop.m2 = 1.0;
    gfc_params par;
    if (gfc_params_default(&par) != GFC_OK) return 1;
    par.n_radial = atoi(argv[3]);
    par.n_angular = atoi(argv[4]);
    gfc_grid grid = {-8.0, 4.0, -4.0, 4.0, m, n};

    double *G = NULL;
    size_t bytes = sizeof(double) * 2 * (size_t)m * (size_t)n;
    if (cudaMalloc((void **)&G, bytes) != cudaSuccess) return 1;
    int rc = gfc_eval_grid(&prop, &par, &grid, G, NULL);
    if (rc != GFC_OK) {
        fprintf(stderr, "gfc_eval_grid: %s (%s)\n", gfc_strerror(rc), gfc_last_error());
        return 1;
    }
    double *h = (double *)malloc(bytes);
    if (!h || cudaMemcpy(h, G, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j)
            printf("%d %d %.17g %.17g\n", i, j, h[2 * (i * n + j)], h[2 * (i * n + j) + 1]);
    gfc_eval_stats st;
    if (gfc_last_stats(&st) != GFC_OK) return 1;
    printf("stats %lld %lld %lld\n", (long long)st.points, (long long)st.node_evals,
           (long long)st.kernel_launches);
    free(h);
    cudaFree(G);
    gfc_release();
    return 0;
}
