// k_chol_f64.cu -- blocked right-looking Cholesky R = L L' in IEEE double
// over a batch of independent instances (one per theta candidate).
//
// The paper factors R by Cholesky on the CPU and by LU on its GPU (Section
// 3); here R is symmetric positive definite, so Cholesky is used throughout.
// Per block column J (tile width NB = 128):
//   potrf:  L_JJ = chol(A_JJ)                    one CTA per instance
//   trsm:   L_IJ = A_IJ L_JJ^-T,  I > J           one CTA per tile
//   update: A_IK -= L_IJ L_KJ^T,  J < K <= I      one CTA per tile
// log|R| = 2 sum log L_ii is accumulated during potrf in a fixed order.
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double* inst_tile(const Batch& b, int t, int I, int J) {
    return b.A + (size_t)t * b.inst_stride + (size_t)tile_index(I, J, b.nt) * GP_TILE_ELEMS;
}

// Factor the diagonal tile of block column J for every live instance.
// Dynamic shared memory: NB*NB doubles.
__global__ void __launch_bounds__(kThreads) k_potrf_f64(Batch b, int J) {
    extern __shared__ double s[];
    __shared__ double inv_piv;
    __shared__ double logs[GP_NB];
    __shared__ int failed;
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    double* T = inst_tile(b, t, J, J);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) s[q] = T[q];
    if (threadIdx.x == 0) failed = -1;
    __syncthreads();
    const int r = threadIdx.x % GP_NB;
    const int h = threadIdx.x / GP_NB;
    for (int c = 0; c < GP_NB; ++c) {
        if (threadIdx.x == 0) {
            double piv = s[c * GP_NB + c];
            if (!(piv > 0.0) || !isfinite(piv)) {
                failed = c;
            } else {
                double l = sqrt(piv);
                s[c * GP_NB + c] = l;
                inv_piv = 1.0 / l;
            }
        }
        __syncthreads();
        if (failed >= 0) break;
        if (h == 0 && r > c) s[c * GP_NB + r] *= inv_piv;
        __syncthreads();
        if (r > c) {
            const double lr = s[c * GP_NB + r];
            for (int k = c + 1 + h; k <= r; k += 2)
                s[k * GP_NB + r] = fma(-lr, s[c * GP_NB + k], s[k * GP_NB + r]);
        }
        __syncthreads();
    }
    if (failed >= 0) {
        if (threadIdx.x == 0) {
            b.st[t].status = GP_ENOTPD;
            b.st[t].fail_col = J * GP_NB + failed;
        }
        return;
    }
    // write back the lower triangle (upper triangle keeps R)
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        int rr = q % GP_NB, cc = q / GP_NB;
        if (rr >= cc) T[q] = s[q];
    }
    // the pivots' logarithms off the serial path, summed in column order
    if (threadIdx.x < GP_NB) logs[threadIdx.x] = log(s[threadIdx.x * GP_NB + threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double logdet = 0.0;
        for (int c = 0; c < GP_NB; ++c) logdet += logs[c];
        b.st[t].logdet += 2.0 * logdet;
    }
}

// L_IJ = A_IJ L_JJ^-T for I = J + 1 + blockIdx.x.  The A tile sits in shared
// memory; column c of X is finished, then removed from the columns after it.
// Column c of L_JJ is read from a two-slot buffer that the second 128
// threads fill one step ahead (the tile plus the buffer stay small enough
// to share an SM with an update CTA).
__global__ void __launch_bounds__(kThreads) k_trsm_f64(Batch b, int J) {
    extern __shared__ double s[];
    __shared__ double inv_diag[GP_NB];
    __shared__ double col[2][GP_NB];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int I = J + 1 + blockIdx.x;
    const double* __restrict__ Ljj = inst_tile(b, t, J, J);
    double* Aij = inst_tile(b, t, I, J);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) s[q] = Aij[q];
    if (threadIdx.x < GP_NB) {
        inv_diag[threadIdx.x] = 1.0 / Ljj[threadIdx.x * GP_NB + threadIdx.x];
        col[0][threadIdx.x] = __ldg(Ljj + threadIdx.x);
    }
    __syncthreads();
    const int r = threadIdx.x % GP_NB;
    const int h = threadIdx.x / GP_NB;
    for (int c = 0; c < GP_NB; ++c) {
        // X[r, c] is final once the previous columns are removed
        const double xrc = s[c * GP_NB + r] * inv_diag[c];
        __syncthreads();
        if (h == 0) s[c * GP_NB + r] = xrc;
        if (h == 1 && c + 1 < GP_NB) col[(c + 1) & 1][r] = __ldg(Ljj + (c + 1) * GP_NB + r);
        const double* Lc = col[c & 1];        // column c of L_JJ (rows k > c below the diagonal)
        for (int k = c + 1 + h; k < GP_NB; k += 2)
            s[k * GP_NB + r] = fma(-xrc, Lc[k], s[k * GP_NB + r]);
        __syncthreads();
    }
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) Aij[q] = s[q];
}

// A_IK -= L_IJ L_KJ^T over the trailing lower triangle of tiles (which =
// kUpdateAll, grid.x = m(m+1)/2 with m = nt - J - 1), its first column K =
// J + 1 (kUpdateColumn, grid.x = m) or the rest (kUpdateRest, grid.x =
// m(m-1)/2); grid.y = instances.
// Thread (tx, ty) of a 16 x 16 layout owns rows tx + 16i and columns
// ty + 16j (i, j < 8) of the 128 x 128 tile.
__global__ void __launch_bounds__(kThreads) k_update_f64(Batch b, int J, int which) {
    constexpr int KC = 16;
    __shared__ double As[KC][GP_NB];
    __shared__ double Bs[KC][GP_NB];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    int ii, kk;
    if (which == kUpdateColumn) {
        ii = blockIdx.x;
        kk = 0;
    } else {
        tri_decode(blockIdx.x, ii, kk);
        if (which == kUpdateRest) {
            ++ii;
            ++kk;
        }
    }
    const int I = J + 1 + ii, K = J + 1 + kk;
    const double* __restrict__ Lij = inst_tile(b, t, I, J);
    const double* __restrict__ Lkj = inst_tile(b, t, K, J);
    double* C = inst_tile(b, t, I, K);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < GP_NB; k0 += KC) {
        __syncthreads();
        for (int q = threadIdx.x; q < KC * GP_NB; q += kThreads) {
            int kq = q / GP_NB, rq = q % GP_NB;
            As[kq][rq] = Lij[(k0 + kq) * GP_NB + rq];
            Bs[kq][rq] = Lkj[(k0 + kq) * GP_NB + rq];
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            double a[8], bb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) bb[j] = Bs[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = ty + 16 * j;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = tx + 16 * i;
            C[c * GP_NB + r] -= acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_potrf_f64(const Batch& b, int J, cudaStream_t s) {
    const size_t smem = GP_TILE_ELEMS * sizeof(double);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_potrf_f64, smem, attr);
    if (e != cudaSuccess) return e;
    k_potrf_f64<<<b.count, kThreads, smem, s>>>(b, J);
    return cudaGetLastError();
}

cudaError_t launch_trsm_f64(const Batch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 1;
    if (m <= 0) return cudaSuccess;
    const size_t smem = GP_TILE_ELEMS * sizeof(double);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_trsm_f64, smem, attr);
    if (e != cudaSuccess) return e;
    k_trsm_f64<<<dim3(m, b.count), kThreads, smem, s>>>(b, J);
    return cudaGetLastError();
}

cudaError_t launch_update_f64(const Batch& b, int J, cudaStream_t s, int which) {
    const int m = b.nt - J - 1;
    const int tiles = which == kUpdateColumn ? m : (which == kUpdateRest ? m * (m - 1) / 2 : m * (m + 1) / 2);
    if (tiles <= 0) return cudaSuccess;
    k_update_f64<<<dim3(tiles, b.count), kThreads, 0, s>>>(b, J, which);
    return cudaGetLastError();
}

}  // namespace gp
