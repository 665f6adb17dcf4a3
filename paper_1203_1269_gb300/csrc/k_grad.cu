// k_grad.cu -- gradient of -2 log L (eq. 4) with respect to theta, in IEEE
// double, for a batch of candidates factored by the FP64 path.
//
//   d(-2logL)/dtheta_k = tr(R^-1 dR_k) - (n / Q) w' dR_k w
//                      = sum_{i != j} M_ij R_ij dlog rho_k(x_i, x_j),
//   M = R^-1 - (n / Q) w w',  w = R^-1 (Y - 1 mu_hat),
//
// from d log|R| = tr(R^-1 dR) and dQ = -w' dR w (mu_hat minimises Q); dR_k
// is zero on the diagonal (the nugget and the unit diagonal do not depend on
// theta).  R^-1 comes from the factor in the tile layout:
//   X = L^-1:   X_JJ = L_JJ^-1, then along tile diagonals s = I - J = 1, 2, ...
//               X_IJ = -X_II sum_{K=J}^{I-1} L_IK X_KJ  (all J of a diagonal at once)
//   R^-1 = X' X:  (R^-1)_IJ = sum_{K >= I} X_KI' X_KJ  (I >= J)
// (n^3/3 more FMAs on the FP64 pipes, like a second factorisation), and one
// pass over the lower tiles recomputes R_ij and dlog rho, reducing d partial
// sums per tile that a last kernel adds in a fixed order.
#include "corr.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double* tile_at(double* base, size_t stride, int t, int I, int J, int nt) {
    return base + (size_t)t * stride + (size_t)tile_index(I, J, nt) * GP_TILE_ELEMS;
}

// acc(r, c) += sum_k opA(A)(r, k) opB(B)(k, c) for one pair of column-major
// 128 x 128 tiles; thread (tx, ty) of a 16 x 16 layout owns rows tx + 16i and
// columns ty + 16j.  TA / TB: use the transpose of A / B.  The operands are
// plain (coherent) loads: k_trtri_step reads a tile it wrote itself.
template <bool TA, bool TB>
__device__ __forceinline__ void tile_mma(double (&acc)[8][8], const double* A, const double* B,
                                         double (*As)[GP_NB], double (*Bs)[GP_NB]) {
    constexpr int KC = 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = 0; k0 < GP_NB; k0 += KC) {
        __syncthreads();
        for (int q = threadIdx.x; q < KC * GP_NB; q += kThreads) {
            // element (row or column index u, k0 + kq), read along the contiguous index
            if (!TA) {
                const int kq = q / GP_NB, u = q % GP_NB;
                As[kq][u] = A[(size_t)(k0 + kq) * GP_NB + u];           // A(u, k)
            } else {
                const int u = q / KC, kq = q % KC;
                As[kq][u] = A[(size_t)u * GP_NB + k0 + kq];             // A(k, u)
            }
            if (!TB) {
                const int u = q / KC, kq = q % KC;
                Bs[kq][u] = B[(size_t)u * GP_NB + k0 + kq];             // B(k, u)
            } else {
                const int kq = q / GP_NB, u = q % GP_NB;
                Bs[kq][u] = B[(size_t)(k0 + kq) * GP_NB + u];           // B(u, k)
            }
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
}

__device__ __forceinline__ void acc_zero(double (&acc)[8][8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
}

__device__ __forceinline__ void acc_store(const double (&acc)[8][8], double* C, double scale) {
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) C[(size_t)(ty + 16 * j) * GP_NB + tx + 16 * i] = scale * acc[i][j];
}

// X_JJ = L_JJ^-1 (lower; zeros above the diagonal), one CTA per (J, instance):
// row i of W from rows j < i, W_ij = -(1/L_ii) sum_{k=j}^{i-1} L_ik W_kj.
// Dynamic smem: L and W as packed lower triangles (row r at r (r + 1) / 2).
constexpr int kPackedTri = GP_NB * (GP_NB + 1) / 2;
__device__ __forceinline__ int prow(int r) { return r * (r + 1) / 2; }

__global__ void __launch_bounds__(kThreads) k_inv_diag(Batch b, double* X) {
    extern __shared__ double sm[];
    double* Lp = sm;
    double* Wp = sm + kPackedTri;
    __shared__ double dinv[GP_NB];
    const int J = blockIdx.x, t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const double* L = tile_at(b.A, b.inst_stride, t, J, J, b.nt);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        const int r = q % GP_NB, c = q / GP_NB;
        if (r >= c) {
            Lp[prow(r) + c] = L[q];
            Wp[prow(r) + c] = 0.0;
        }
        if (r == c) dinv[r] = 1.0 / L[q];    // one division per pivot
    }
    __syncthreads();
    for (int i = 0; i < GP_NB; ++i) {
        const double inv = dinv[i];
        for (int j = threadIdx.x; j < i; j += kThreads) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s = fma(Lp[prow(i) + k], Wp[prow(k) + j], s);
            Wp[prow(i) + j] = -inv * s;
        }
        if (threadIdx.x == 0) Wp[prow(i) + i] = inv;
        __syncthreads();
    }
    double* Xt = tile_at(X, b.inst_stride, t, J, J, b.nt);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        const int r = q % GP_NB, c = q / GP_NB;
        Xt[q] = (r >= c) ? Wp[prow(r) + c] : 0.0;
    }
}

// Tile diagonal s of X = L^-1: X_IJ, I = J + s, for J = blockIdx.x.
__global__ void __launch_bounds__(kThreads) k_trtri_step(Batch b, double* X, int s) {
    __shared__ double As[16][GP_NB];
    __shared__ double Bs[16][GP_NB];
    const int J = blockIdx.x, t = blockIdx.y, I = J + s, nt = b.nt;
    if (b.st[t].status != GP_OK) return;
    double acc[8][8];
    acc_zero(acc);
    for (int K = J; K < I; ++K)
        tile_mma<false, false>(acc, tile_at(b.A, b.inst_stride, t, I, K, nt),
                               tile_at(X, b.inst_stride, t, K, J, nt), As, Bs);
    double* Xij = tile_at(X, b.inst_stride, t, I, J, nt);
    __syncthreads();
    acc_store(acc, Xij, 1.0);                 // S = sum_K L_IK X_KJ, for the product below
    __syncthreads();
    acc_zero(acc);
    tile_mma<false, false>(acc, tile_at(X, b.inst_stride, t, I, I, nt), Xij, As, Bs);
    __syncthreads();                          // every read of S is done
    acc_store(acc, Xij, -1.0);
}

// (R^-1)_IJ = sum_{K >= I} X_KI' X_KJ for the lower tile q = blockIdx.x.
__global__ void __launch_bounds__(kThreads) k_lauum(Batch b, const double* X, double* Ri) {
    __shared__ double As[16][GP_NB];
    __shared__ double Bs[16][GP_NB];
    const int t = blockIdx.y, nt = b.nt;
    if (b.st[t].status != GP_OK) return;
    int J = 0;
    {
        long long rem = blockIdx.x;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(blockIdx.x - tile_index(J, J, nt));
    double acc[8][8];
    acc_zero(acc);
    for (int K = I; K < nt; ++K)
        tile_mma<true, false>(acc, tile_at(const_cast<double*>(X), b.inst_stride, t, K, I, nt),
                              tile_at(const_cast<double*>(X), b.inst_stride, t, K, J, nt), As, Bs);
    acc_store(acc, tile_at(Ri, b.inst_stride, t, I, J, nt), 1.0);
}

// e = b - mu_hat a in column 1 of Z (w = L^-T e follows by the backward solve)
__global__ void k_residual_vec(Batch b, double* Z, size_t zs) {
    const int t = blockIdx.x;
    const InstState st = b.st[t];
    if (st.status != GP_OK) return;
    const int npad = b.nt * GP_NB;
    double* z0 = Z + (size_t)t * zs;
    double* z1 = z0 + npad;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) z1[i] = fma(-st.mu, z0[i], z1[i]);
}

// Partial sums of sum_{i != j} M_ij R_ij dlog rho_k over lower tile
// q = blockIdx.x (both (i, j) and (j, i): twice the strictly lower part).
// D_k = |dx_k|^p (power-exponential) or |dx_k| (Matern) is taken once per
// element and serves both R_ij and its derivative:
//   dlog rho_k / dtheta_k = -D_k                       (eq. 2, Matern 1/2)
//                         = -h / (1 + h) c D_k          (3/2, h = c theta_k D_k)
//                         = -h (1 + h) / (3 + 3h + h^2) c D_k   (5/2)
template <int DB>
__global__ void __launch_bounds__(kThreads) k_grad_tiles(Batch b, const double* Ri, const double* Z, size_t zs,
                                                         double* partial, int ntiles) {
    __shared__ double red[kThreads / 32][DB];
    const int t = blockIdx.y, nt = b.nt, n = b.n, d = b.d;
    const InstState st = b.st[t];
    if (st.status != GP_OK) return;
    int J = 0;
    {
        long long rem = blockIdx.x;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(blockIdx.x - tile_index(J, J, nt));
    const double* R1 = tile_at(const_cast<double*>(Ri), b.inst_stride, t, I, J, nt);
    const double* w = Z + (size_t)t * zs + (size_t)nt * GP_NB;
    const double* th = b.theta + (size_t)t * d;
    const double nq = n / st.Q;
    const int corr = b.corr;
    const bool matern = corr_is_matern(corr);
    const double cm = corr_theta_scale(corr);
    double acc[DB];
#pragma unroll
    for (int k = 0; k < DB; ++k) acc[k] = 0.0;
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        const int r = q % GP_NB, c = q / GP_NB;
        const int gi = I * GP_NB + r, gj = J * GP_NB + c;
        if (gi >= n || gj >= n || gi <= gj) continue;
        const double m = R1[q] - nq * w[gi] * w[gj];
        double D[DB], h[DB];
        double s = 0.0, qp = 1.0;
#pragma unroll
        for (int k = 0; k < DB; ++k) {
            D[k] = 0.0;
            h[k] = 0.0;
            if (k < d) {
                const double a = fabs(b.x[(size_t)gi * d + k] - b.x[(size_t)gj * d + k]);
                D[k] = matern ? a : ((b.p == 2.0) ? a * a : (b.p == 1.0 ? a : (a == 0.0 ? 0.0 : pow(a, b.p))));
                h[k] = cm * th[k] * D[k];
                s += h[k];
                if (matern) qp *= matern_q(h[k], corr);
            }
        }
        const double mr = 2.0 * m * qp * exp(-s);
#pragma unroll
        for (int k = 0; k < DB; ++k) {
            if (k < d) {
                double dl = -D[k];
                if (corr == GP_CORR_MATERN32) dl = -h[k] / (1.0 + h[k]) * cm * D[k];
                if (corr == GP_CORR_MATERN52) dl = -h[k] * (1.0 + h[k]) / (3.0 + 3.0 * h[k] + h[k] * h[k]) * cm * D[k];
                acc[k] = fma(mr, dl, acc[k]);
            }
        }
    }
    // fixed-order block reduction of the d sums
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < DB; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < d) {
        double v = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) v += red[i][threadIdx.x];
        partial[((size_t)t * ntiles + blockIdx.x) * d + threadIdx.x] = v;
    }
}

// grad[t][k] = sum over tiles, in tile order; NaN where the likelihood
// itself failed (status: the finalize kernel's, which also flags Q = 0)
__global__ void k_grad_reduce(Batch b, const double* partial, int ntiles, const int* status, double* grad) {
    const int t = blockIdx.x, d = b.d;
    const int k = threadIdx.x;
    if (k >= d) return;
    if (b.st[t].status != GP_OK || status[t] != GP_OK) {
        grad[(size_t)t * d + k] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double v = 0.0;
    for (int q = 0; q < ntiles; ++q) v += partial[((size_t)t * ntiles + q) * d + k];
    grad[(size_t)t * d + k] = v;
}

}  // namespace

cudaError_t launch_grad(const Batch& b, double* Z, size_t zs, double* X, double* Ri, double* partial,
                        const int* status, double* grad, cudaStream_t s, int* kernels) {
    const int nt = b.nt;
    const int ntiles = (int)packed_tiles(nt);
    int k = 0;
    k_residual_vec<<<b.count, kThreads, 0, s>>>(b, Z, zs);
    ++k;
    cudaError_t e = launch_backward_solve(b, Z, zs, 1, s);   // w = L^-T (b - mu a)
    if (e != cudaSuccess) return e;
    ++k;
    {
        const size_t smem = (size_t)2 * kPackedTri * sizeof(double);
        static std::atomic<size_t> attr[kMaxDevices];
        e = raise_smem_limit(k_inv_diag, smem, attr);
        if (e != cudaSuccess) return e;
        k_inv_diag<<<dim3(nt, b.count), kThreads, smem, s>>>(b, X);
        ++k;
    }
    for (int st = 1; st < nt; ++st) {
        k_trtri_step<<<dim3(nt - st, b.count), kThreads, 0, s>>>(b, X, st);
        ++k;
    }
    k_lauum<<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, X, Ri);
    ++k;
    if (b.d <= 4)
        k_grad_tiles<4><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, Ri, Z, zs, partial, ntiles);
    else if (b.d <= 8)
        k_grad_tiles<8><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, Ri, Z, zs, partial, ntiles);
    else
        k_grad_tiles<16><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, Ri, Z, zs, partial, ntiles);
    ++k;
    k_grad_reduce<<<b.count, 64, 0, s>>>(b, partial, ntiles, status, grad);
    ++k;
    if (kernels) *kernels = k;
    return cudaGetLastError();
}

}  // namespace gp
