// k_grad.cu -- gradient of -2 log L (eq. 4) with respect to theta for a
// batch of candidates factored by the FP64 path.
//
//   d(-2logL)/dtheta_k = tr(R^-1 dR_k) - (n / Q) w' dR_k w
//                      = sum_{i != j} M_ij R_ij dlog rho_k(x_i, x_j),
//   M = R^-1 - (n / Q) w w',  w = R^-1 (Y - 1 mu_hat),
//
// from d log|R| = tr(R^-1 dR) and dQ = -w' dR w (mu_hat minimises Q); dR_k
// is zero on the diagonal (the nugget and the unit diagonal do not depend on
// theta).  -2logL and w come from the IEEE-double factor; R^-1 is formed
// from it in double-float on the FP32 pipes (n^3/3 multiply-adds, which on
// the FP64 pipes would cost more than the factorisation itself):
//   X = L^-1:   X_JJ = L_JJ^-1 (double, in shared memory), then along tile
//               diagonals s = I - J = 1, 2, ...
//               X_IJ = -X_II sum_{K=J}^{I-1} L_IK X_KJ  (all J of a diagonal at
//               once, in 64 x 64 quadrants, the sum staged in the R^-1 buffer)
//   R^-1 = X' X:  (R^-1)_IJ = sum_{K >= I} X_KI' X_KJ  (I >= J)
// The factor is rewritten in place as double-float once the likelihood is
// done (8 bytes either way), so every tile operand is a float pair.  One pass
// over the lower tiles then recomputes R_ij (powers in double-float, as the
// assembly takes them) and dlog rho, reducing d partial sums per tile that a
// last kernel adds in a fixed order.
#include "corr.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T* tile_at(T* base, size_t stride, int t, int I, int J, int nt) {
    return base + (size_t)t * stride + (size_t)tile_index(I, J, nt) * GP_TILE_ELEMS;
}

// acc(r, c) += sum_k opA(A)(r, k) opB(B)(k, c) for one pair of column-major
// 128 x 128 double-float tiles; thread (tx, ty) of a 16 x 16 layout owns
// rows tx + 16i and columns ty + 16j.  TA / TB: use the transpose of A / B.
// The operands are plain (coherent) loads.
template <bool TA, bool TB>
__device__ __forceinline__ void tile_mma(dfl (&acc)[8][8], const float2* A, const float2* B,
                                         dfl (*As)[GP_NB], dfl (*Bs)[GP_NB]) {
    constexpr int KC = 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = 0; k0 < GP_NB; k0 += KC) {
        __syncthreads();
        for (int q = threadIdx.x; q < KC * GP_NB; q += kThreads) {
            // element (row or column index u, k0 + kq), read along the contiguous index
            float2 a, bv;
            int ka, ua, kb, ub;
            if (!TA) {
                ka = q / GP_NB; ua = q % GP_NB;
                a = A[(size_t)(k0 + ka) * GP_NB + ua];          // A(u, k)
            } else {
                ua = q / KC; ka = q % KC;
                a = A[(size_t)ua * GP_NB + k0 + ka];            // A(k, u)
            }
            if (!TB) {
                ub = q / KC; kb = q % KC;
                bv = B[(size_t)ub * GP_NB + k0 + kb];           // B(k, u)
            } else {
                kb = q / GP_NB; ub = q % GP_NB;
                bv = B[(size_t)(k0 + kb) * GP_NB + ub];         // B(u, k)
            }
            As[ka][ua] = dfl{a.x, a.y};
            Bs[kb][ub] = dfl{bv.x, bv.y};
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < KC; ++k) {
            dfl a[8], bb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) bb[j] = Bs[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = df_fma(a[i], bb[j], acc[i][j]);
        }
    }
}

__device__ __forceinline__ void acc_zero(dfl (&acc)[8][8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = dfl{0.f, 0.f};
}

__device__ __forceinline__ void acc_store(const dfl (&acc)[8][8], float2* C, bool negate) {
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const dfl v = negate ? df_neg(acc[i][j]) : acc[i][j];
            C[(size_t)(ty + 16 * j) * GP_NB + tx + 16 * i] = make_float2(v.hi, v.lo);
        }
}

// The factor, rewritten in place as double-float (hi, lo) pairs.
__global__ void k_factor_to_df(Batch b, size_t elems) {
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    double* A = b.A + (size_t)t * b.inst_stride;
    float2* F = reinterpret_cast<float2*>(A);
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < elems; q += (size_t)gridDim.x * blockDim.x) {
        const dfl v = df_from_double(A[q]);
        F[q] = make_float2(v.hi, v.lo);
    }
}

// X_JJ = L_JJ^-1 (lower; zeros above the diagonal), one CTA per (J, instance),
// in double: row i of W from rows j < i, W_ij = -(1/L_ii) sum_{k=j}^{i-1} L_ik W_kj.
// Dynamic smem: L and W as packed lower triangles (row r at r (r + 1) / 2).
constexpr int kPackedTri = GP_NB * (GP_NB + 1) / 2;
__device__ __forceinline__ int prow(int r) { return r * (r + 1) / 2; }

__global__ void __launch_bounds__(kThreads) k_inv_diag(Batch b, const float2* L2, float2* X) {
    extern __shared__ double sm[];
    double* Lp = sm;
    double* Wp = sm + kPackedTri;
    __shared__ double dinv[GP_NB];
    const int J = blockIdx.x, t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const float2* L = tile_at(L2, b.inst_stride, t, J, J, b.nt);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        const int r = q % GP_NB, c = q / GP_NB;
        if (r >= c) {
            const float2 v = L[q];
            const double l = (double)v.x + (double)v.y;
            Lp[prow(r) + c] = l;
            Wp[prow(r) + c] = 0.0;
            if (r == c) dinv[r] = 1.0 / l;    // one division per pivot
        }
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
    float2* Xt = tile_at(X, b.inst_stride, t, J, J, b.nt);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
        const int r = q % GP_NB, c = q / GP_NB;
        const dfl v = (r >= c) ? df_from_double(Wp[prow(r) + c]) : dfl{0.f, 0.f};
        Xt[q] = make_float2(v.hi, v.lo);
    }
}

// Quadrant products for the tile diagonals of X = L^-1: a CTA forms one
// 64 x 64 quadrant (qr, qc) of a 128 x 128 output tile, thread (tx, ty) of a
// 16 x 16 layout rows tx + 16i and columns ty + 16j (4 x 4), so that a tile
// diagonal spreads over four times as many CTAs as tiles: a single
// candidate's inverse is a chain of nt - 1 such steps.
// acc(r, c) += sum_k A(64 qr + r, k) B(k, 64 qc + c) for column-major tiles.
__device__ __forceinline__ void quad_mma(dfl (&acc)[4][4], const float2* A, const float2* B, int qr, int qc,
                                         dfl (*As)[64], dfl (*Bs)[64]) {
    constexpr int KC = 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = 0; k0 < GP_NB; k0 += KC) {
        __syncthreads();
        for (int q = threadIdx.x; q < KC * 64; q += kThreads) {
            {
                const int kq = q / 64, u = q % 64;                   // A(64 qr + u, k0 + kq)
                const float2 a = A[(size_t)(k0 + kq) * GP_NB + 64 * qr + u];
                As[kq][u] = dfl{a.x, a.y};
            }
            {
                const int u = q / KC, kq = q % KC;                   // B(k0 + kq, 64 qc + u)
                const float2 v = B[(size_t)(64 * qc + u) * GP_NB + k0 + kq];
                Bs[kq][u] = dfl{v.x, v.y};
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            dfl a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = df_fma(a[i], bb[j], acc[i][j]);
        }
    }
}

__device__ __forceinline__ void quad_store(const dfl (&acc)[4][4], float2* C, int qr, int qc, bool negate) {
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const dfl v = negate ? df_neg(acc[i][j]) : acc[i][j];
            C[(size_t)(64 * qc + ty + 16 * j) * GP_NB + 64 * qr + tx + 16 * i] = make_float2(v.hi, v.lo);
        }
}

// Tile diagonal s of X = L^-1, first half: S_IJ = sum_{K=J}^{I-1} L_IK X_KJ
// (I = J + s, J = blockIdx.x, quadrant blockIdx.z) into S (the R^-1 buffer,
// free until k_lauum).
__global__ void __launch_bounds__(kThreads) k_trtri_sum(Batch b, const float2* L2, const float2* X, float2* S, int s) {
    __shared__ dfl As[16][64];
    __shared__ dfl Bs[16][64];
    const int J = blockIdx.x, t = blockIdx.y, I = J + s, nt = b.nt;
    const int qr = blockIdx.z & 1, qc = blockIdx.z >> 1;
    if (b.st[t].status != GP_OK) return;
    dfl acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = dfl{0.f, 0.f};
    for (int K = J; K < I; ++K)
        quad_mma(acc, tile_at(L2, b.inst_stride, t, I, K, nt), tile_at(X, b.inst_stride, t, K, J, nt), qr, qc, As, Bs);
    quad_store(acc, tile_at(S, b.inst_stride, t, I, J, nt), qr, qc, false);
}

// Second half: X_IJ = -X_II S_IJ.
__global__ void __launch_bounds__(kThreads) k_trtri_apply(Batch b, float2* X, const float2* S, int s) {
    __shared__ dfl As[16][64];
    __shared__ dfl Bs[16][64];
    const int J = blockIdx.x, t = blockIdx.y, I = J + s, nt = b.nt;
    const int qr = blockIdx.z & 1, qc = blockIdx.z >> 1;
    if (b.st[t].status != GP_OK) return;
    dfl acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = dfl{0.f, 0.f};
    quad_mma(acc, tile_at(X, b.inst_stride, t, I, I, nt), tile_at(S, b.inst_stride, t, I, J, nt), qr, qc, As, Bs);
    quad_store(acc, tile_at(X, b.inst_stride, t, I, J, nt), qr, qc, true);
}

// (R^-1)_IJ = sum_{K >= I} X_KI' X_KJ for the lower tile q = blockIdx.x.
__global__ void __launch_bounds__(kThreads, 1) k_lauum(Batch b, const float2* X, float2* Ri) {
    __shared__ dfl As[16][GP_NB];
    __shared__ dfl Bs[16][GP_NB];
    const int t = blockIdx.y, nt = b.nt;
    if (b.st[t].status != GP_OK) return;
    int J = 0;
    {
        long long rem = blockIdx.x;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(blockIdx.x - tile_index(J, J, nt));
    dfl acc[8][8];
    acc_zero(acc);
    for (int K = I; K < nt; ++K)
        tile_mma<true, false>(acc, tile_at(X, b.inst_stride, t, K, I, nt), tile_at(X, b.inst_stride, t, K, J, nt),
                              As, Bs);
    acc_store(acc, tile_at(Ri, b.inst_stride, t, I, J, nt), false);
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
__global__ void __launch_bounds__(kThreads) k_grad_tiles(Batch b, const float2* Ri, const double* Z, size_t zs,
                                                         double* partial, int ntiles) {
    __shared__ double red[kThreads / 32][DB];
    __shared__ dfl tab[kExpTab];
    fill_exp2_table(tab);
    __syncthreads();
    const int t = blockIdx.y, nt = b.nt, n = b.n, d = b.d;
    const InstState st = b.st[t];
    if (st.status != GP_OK) return;
    int J = 0;
    {
        long long rem = blockIdx.x;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(blockIdx.x - tile_index(J, J, nt));
    const float2* R1 = tile_at(Ri, b.inst_stride, t, I, J, nt);
    const int pmode = pow_mode(b.p);
    const dfl pd = df_from_double(b.p);
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
        const double m = ((double)R1[q].x + (double)R1[q].y) - nq * w[gi] * w[gj];
        double D[DB], h[DB];
        double s = 0.0, qp = 1.0;
#pragma unroll
        for (int k = 0; k < DB; ++k) {
            D[k] = 0.0;
            h[k] = 0.0;
            if (k < d) {
                const double a = fabs(b.x[(size_t)gi * d + k] - b.x[(size_t)gj * d + k]);
                // |dx|^p for general p in double-float (FP64 pow is scarce here)
                D[k] = (matern || pmode == kPowOne) ? a
                                                    : (pmode == kPowTwo ? a * a
                                                                        : df_to_double(df_powabs(df_from_double(a), pmode, b.p, pd, tab)));
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
    cudaError_t e = launch_backward_solve(b, Z, zs, 1, s);   // w = L^-T (b - mu a), double factor
    if (e != cudaSuccess) return e;
    k += solve_f64_launches(nt, true);
    // from here on the factor, X and R^-1 are double-float tiles
    const size_t elems = (size_t)ntiles * GP_TILE_ELEMS;
    k_factor_to_df<<<dim3(64, b.count), kThreads, 0, s>>>(b, elems);
    ++k;
    const float2* L2 = reinterpret_cast<const float2*>(b.A);
    float2* X2 = reinterpret_cast<float2*>(X);
    float2* R2 = reinterpret_cast<float2*>(Ri);
    {
        const size_t smem = (size_t)2 * kPackedTri * sizeof(double);
        static std::atomic<size_t> attr[kMaxDevices];
        e = raise_smem_limit(k_inv_diag, smem, attr);
        if (e != cudaSuccess) return e;
        k_inv_diag<<<dim3(nt, b.count), kThreads, smem, s>>>(b, L2, X2);
        ++k;
    }
    for (int st = 1; st < nt; ++st) {
        k_trtri_sum<<<dim3(nt - st, b.count, 4), kThreads, 0, s>>>(b, L2, X2, R2, st);
        k_trtri_apply<<<dim3(nt - st, b.count, 4), kThreads, 0, s>>>(b, X2, R2, st);
        k += 2;
    }
    k_lauum<<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, X2, R2);
    ++k;
    if (b.d <= 4)
        k_grad_tiles<4><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, R2, Z, zs, partial, ntiles);
    else if (b.d <= 8)
        k_grad_tiles<8><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, R2, Z, zs, partial, ntiles);
    else
        k_grad_tiles<16><<<dim3(ntiles, b.count), kThreads, 0, s>>>(b, R2, Z, zs, partial, ntiles);
    ++k;
    k_grad_reduce<<<b.count, 64, 0, s>>>(b, partial, ntiles, status, grad);
    ++k;
    if (kernels) *kernels = k;
    return cudaGetLastError();
}

}  // namespace gp
