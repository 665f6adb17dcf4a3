// gp_internal.cuh -- shared definitions of libgp's CUDA sources.
//
// Storage of R and of its Cholesky factor (per instance): the lower
// triangle in NB x NB tiles.  Tile (I, J), I >= J, starts at tile index
// J*nt - J*(J-1)/2 + (I - J) (tile columns packed one after another), and
// is column-major inside (element (r, c) at r + NB*c).  Rows/columns >= n
// hold the identity so that the padded factor is block-diag(L, I).
// Diagonal tiles hold both triangles of R; after factorisation their
// lower triangle holds L.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/gp.h"

#define GP_NB 128
#define GP_TILE_ELEMS (GP_NB * GP_NB)
#define GP_MAX_D 64

namespace gp {

__host__ __device__ inline int num_tiles(int n) { return (n + GP_NB - 1) / GP_NB; }

__host__ __device__ inline long long tile_index(int I, int J, int nt) {
    return (long long)J * nt - (long long)J * (J - 1) / 2 + (I - J);
}

__host__ __device__ inline long long packed_tiles(int nt) {
    return (long long)nt * (nt + 1) / 2;
}

__host__ __device__ inline size_t packed_elems(int n) {
    int nt = num_tiles(n);
    return (size_t)packed_tiles(nt) * GP_TILE_ELEMS;
}

// lower-triangle linear index q -> (i, k), k <= i, over an m x m triangle
__device__ inline void tri_decode(int q, int& i, int& k) {
    int r = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((long long)(r + 1) * (r + 2) / 2 <= q) ++r;
    while ((long long)r * (r + 1) / 2 > q) --r;
    i = r;
    k = q - r * (r + 1) / 2;
}

// Per-instance record written by the factorisation and solve kernels.
struct InstState {
    double logdet;
    double aa;      // 1'R^-1 1
    double ab;      // 1'R^-1 Y
    double mu;
    double Q;
    double bb;
    int status;
    int fail_col;
};

// Batched problem description handed to the kernels (by value).
struct Batch {
    int n, d, nt, count;          // count = instances in this launch chunk
    double p, delta;
    const double* x;              // n x d
    const double* y;              // n
    const double* theta;          // count x d (already offset to the chunk)
    double* A;                    // count * packed_elems(n)
    size_t inst_stride;           // elements between instances in A
    InstState* st;                // count
};

// ---- kernels (launch helpers, all on `stream`) ----------------------------
cudaError_t launch_validate_theta(const Batch& b, cudaStream_t s);
cudaError_t launch_assemble_tiles(const Batch& b, cudaStream_t s);
cudaError_t launch_assemble_dense(int n, int d, const double* x, const double* theta, double p,
                                  double delta, double* R, cudaStream_t s);
cudaError_t launch_potrf_f64(const Batch& b, int J, cudaStream_t s);
cudaError_t launch_trsm_f64(const Batch& b, int J, cudaStream_t s);
cudaError_t launch_update_f64(const Batch& b, int J, cudaStream_t s);
cudaError_t launch_forward_solve(const Batch& b, double* Z, size_t z_stride, cudaStream_t s);
cudaError_t launch_finalize(const Batch& b, const double* Z, size_t z_stride, double* nll,
                            double* mu, double* sigma2, double* logdet, int* status,
                            cudaStream_t s);
cudaError_t launch_fit_finish(const Batch& b, double* Z, size_t z_stride, double* scalars,
                              cudaStream_t s);
cudaError_t launch_backward_solve(const Batch& b, double* Z, size_t z_stride, int col,
                                  cudaStream_t s);
cudaError_t launch_predict(int n, int d, int nt, const double* x, const double* theta, double p,
                           double c0, const double* L, const double* w, const double* a,
                           const double* scalars, int N, const double* xs, double* yhat,
                           double* s2, double* work, int chunk, cudaStream_t s);

}  // namespace gp
