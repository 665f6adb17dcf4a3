// k_solve.cu -- triangular solves with the tiled factor and the profile
// estimates of Section 2.
//
// forward:  [a b] = L^-1 [1 Y]        (two right-hand sides at once)
// finalize: 1'R^-1 1 = a'a, 1'R^-1 Y = a'b, mu_hat = a'b / a'a      (eq. 3)
//           e = b - mu_hat a = L^-1 (Y - 1 mu_hat), Q = e'e,
//           sigma2_hat = Q / n                                       (eq. 3)
//           -2logL = log|R| + n log Q                                (eq. 4)
// backward: w = L^-T z  (for the kriging weights R^-1 (Y - 1 mu_hat))
//
// Z holds, per instance, two columns of length npad = nt*NB: Z[0..npad) and
// Z[npad..2 npad).  The solves are tile-parallel (below); every reduction
// runs in a fixed order, so results do not depend on what else is in the
// batch.
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ const double* tile_ptr(const Batch& b, int t, int I, int J) {
    return b.A + (size_t)t * b.inst_stride + (size_t)tile_index(I, J, b.nt) * GP_TILE_ELEMS;
}

// Block-wide sum in a fixed order (warp shuffles, then warp 0).
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// The triangular solves are tile-parallel, one launch per block column (so
// that a single instance, as gp_fit has, still spreads its factor over
// every SM): a diagonal step per instance solves with the diagonal tile,
// staged in shared memory, and a tile step subtracts the products of the
// next tiles from the right-hand sides in Z, every tile of the block column
// at once, one CTA per tile.  A block's right-hand side takes the products
// in block-column order, so the results are the same bits at any batch size.
constexpr int kTileThreads = 1024;
constexpr int kDiagStride = GP_NB + 1;        // staged diagonal tile: D[c * kDiagStride + r] = L_rc
constexpr size_t kDiagSmem = (size_t)GP_NB * kDiagStride * sizeof(double);

__device__ __forceinline__ void stage_diag(const double* L, double* D) {
    for (int e = threadIdx.x; e < GP_TILE_ELEMS; e += blockDim.x) D[(e >> 7) * kDiagStride + (e & 127)] = __ldg(L + e);
}

// Z <- [1 Y] (padded rows zero), the forward solve's right-hand sides
__global__ void k_rhs_f64(Batch b, double* Z, size_t zs) {
    const int npad = b.nt * GP_NB;
    double* z0 = Z + (size_t)blockIdx.y * zs;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
        const bool in = i < b.n;
        z0[i] = in ? 1.0 : 0.0;
        z0[npad + i] = in ? b.y[i] : 0.0;
    }
}

// Forward, block J, one instance per CTA (256 threads: thread (r, k) owns
// row r of right-hand side k): Z_J holds [1 Y]_J less the products of the
// tiles left of it; L_JJ z = Z_J by columns, x_c = v_c (1 / L_cc), then
// v_r -= L_rc x_c for r > c.  Row c's owner publishes x_c before the one
// barrier of step c; every other value stays in its owner's register.
__global__ void __launch_bounds__(2 * GP_NB) k_fwd_diag_f64(Batch b, double* Z, size_t zs, int J) {
    extern __shared__ double D[];
    __shared__ double xc[2][GP_NB];
    __shared__ double inv[GP_NB];
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    stage_diag(tile_ptr(b, t, J, J), D);
    const int r = threadIdx.x & (GP_NB - 1), k = threadIdx.x >> 7;
    double* z = Z + (size_t)t * zs + (size_t)k * b.nt * GP_NB + (size_t)J * GP_NB;
    double v = z[r];
    __syncthreads();
    if (k == 0) inv[r] = 1.0 / D[r * kDiagStride + r];
    __syncthreads();
    for (int c = 0; c < GP_NB; ++c) {
        if (r == c) {
            v *= inv[c];
            xc[k][c] = v;
        }
        __syncthreads();
        if (r > c) v = fma(-D[c * kDiagStride + r], xc[k][c], v);
    }
    z[r] = v;
}

// Forward, tiles (I, J), I > J, one CTA each (1024 threads: thread (r, g)
// takes columns 16 g .. 16 g + 15 of row r): Z_I -= L_IJ z_J, the 8 column
// parts added in order.
__global__ void __launch_bounds__(kTileThreads) k_fwd_tiles_f64(Batch b, double* Z, size_t zs, int J) {
    __shared__ double xs[2][GP_NB];
    __shared__ double part[8][2][GP_NB];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int I = J + 1 + blockIdx.x;
    const int npad = b.nt * GP_NB;
    double* z0 = Z + (size_t)t * zs;
    const int tid = threadIdx.x;
    if (tid < 2 * GP_NB) xs[tid >> 7][tid & 127] = z0[(size_t)(tid >> 7) * npad + (size_t)J * GP_NB + (tid & 127)];
    __syncthreads();
    const double* L = tile_ptr(b, t, I, J);
    const int r = tid & (GP_NB - 1), g = tid >> 7;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int c = 16 * g; c < 16 * g + 16; ++c) {
        const double l = __ldg(L + (size_t)c * GP_NB + r);
        a0 = fma(l, xs[0][c], a0);
        a1 = fma(l, xs[1][c], a1);
    }
    part[g][0][r] = a0;
    part[g][1][r] = a1;
    __syncthreads();
    if (tid < 2 * GP_NB) {
        const int k = tid >> 7;
        double s = part[0][k][r];
#pragma unroll
        for (int q = 1; q < 8; ++q) s += part[q][k][r];
        double* zi = z0 + (size_t)k * npad + (size_t)I * GP_NB + r;
        *zi -= s;
    }
}

// Backward, block I of column col, one instance per CTA (128 threads, one
// row each): Z_I holds z_I less the products of the tiles below it;
// L_II^T w = Z_I from the last column back, x_c = v_c (1 / L_cc), then
// v_r -= L_cr x_c for r < c.
__global__ void __launch_bounds__(GP_NB) k_bwd_diag_f64(Batch b, double* Z, size_t zs, int col, int I) {
    extern __shared__ double D[];
    __shared__ double xc[GP_NB];
    __shared__ double inv[GP_NB];
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    stage_diag(tile_ptr(b, t, I, I), D);
    const int r = threadIdx.x;
    double* z = Z + (size_t)t * zs + (size_t)col * b.nt * GP_NB + (size_t)I * GP_NB;
    double v = z[r];
    __syncthreads();
    inv[r] = 1.0 / D[r * kDiagStride + r];
    __syncthreads();
    for (int c = GP_NB - 1; c >= 0; --c) {
        if (r == c) {
            v *= inv[c];
            xc[c] = v;
        }
        __syncthreads();
        if (r < c) v = fma(-D[r * kDiagStride + c], xc[c], v);
    }
    z[r] = v;
}

// Backward, tiles (I, K), K < I, one CTA each (32 warps: warp w takes
// columns w, w + 32, w + 64, w + 96, lane l rows l, l + 32, l + 64, l + 96,
// then a shuffle sum): Z_K -= L_IK^T w_I.
__global__ void __launch_bounds__(kTileThreads) k_bwd_tiles_f64(Batch b, double* Z, size_t zs, int col, int I) {
    __shared__ double ws[GP_NB];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int K = blockIdx.x;
    double* z = Z + (size_t)t * zs + (size_t)col * b.nt * GP_NB;
    if (threadIdx.x < GP_NB) ws[threadIdx.x] = z[(size_t)I * GP_NB + threadIdx.x];
    __syncthreads();
    const double* L = tile_ptr(b, t, I, K);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double s[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double* Lc = L + (size_t)(w + 32 * q) * GP_NB;
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fma(__ldg(Lc + lane + 32 * j), ws[lane + 32 * j], a);
        s[q] = a;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double a = s[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) z[(size_t)K * GP_NB + w + 32 * q] -= a;
    }
}

// Reductions and the likelihood for one instance per CTA.
// Q is treated as zero when Q <= 16 n u^2 b'b (u = 2^-53): e = b - mu a then
// holds only rounding noise (Y in the span of 1, always so for n = 1).
__global__ void __launch_bounds__(kThreads) k_finalize(Batch b, const double* Z, size_t zs,
                                                       double* nll, double* mu, double* sigma2,
                                                       double* logdet, int* status) {
    __shared__ double red[kThreads / 32];
    const int t = blockIdx.x;
    InstState st = b.st[t];
    const int n = b.n;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (st.status != GP_OK) {
        if (threadIdx.x == 0) {
            nll[t] = (st.status == GP_ENOTPD) ? __longlong_as_double(0x7ff0000000000000LL) : nan;
            mu[t] = nan;
            sigma2[t] = nan;
            if (logdet) logdet[t] = nan;
            status[t] = st.status;
        }
        return;
    }
    const int npad = b.nt * GP_NB;
    const double* a = Z + (size_t)t * zs;
    const double* bv = a + npad;
    double saa = 0.0, sab = 0.0, sbb = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double ai = a[i], bi = bv[i];
        saa = fma(ai, ai, saa);
        sab = fma(ai, bi, sab);
        sbb = fma(bi, bi, sbb);
    }
    const double aa = block_sum(saa, red);
    const double ab = block_sum(sab, red);
    const double bb = block_sum(sbb, red);
    const double m = ab / aa;
    double sq = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double e = fma(-m, a[i], bv[i]);
        sq = fma(e, e, sq);
    }
    const double Q = block_sum(sq, red);
    if (threadIdx.x == 0) {
        const double u = 1.1102230246251565e-16;
        const bool degenerate = Q <= 16.0 * n * u * u * bb;
        const double ld = st.logdet;
        nll[t] = degenerate ? -__longlong_as_double(0x7ff0000000000000LL) : ld + n * log(Q);
        mu[t] = m;
        sigma2[t] = Q / n;
        if (logdet) logdet[t] = ld;
        status[t] = degenerate ? GP_EDEGENERATE : GP_OK;
        st.aa = aa; st.ab = ab; st.bb = bb; st.mu = m; st.Q = Q;
        b.st[t] = st;
    }
}

// After finalize: scalars[4] = Q, scalars[5] = a'a, and column 1 of Z
// becomes e = b - mu_hat a = L^-1 (Y - 1 mu_hat), ready for the backward
// solve that gives the kriging weights w = R^-1 (Y - 1 mu_hat).
__global__ void k_fit_finish(Batch b, double* Z, size_t zs, double* scalars) {
    const int t = blockIdx.x;
    const InstState st = b.st[t];
    if (st.status != GP_OK) return;
    const int npad = b.nt * GP_NB;
    double* z0 = Z + (size_t)t * zs;
    double* z1 = z0 + npad;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) z1[i] = fma(-st.mu, z0[i], z1[i]);
    if (threadIdx.x == 0) {
        scalars[4] = st.Q;
        scalars[5] = st.aa;
    }
}

}  // namespace

cudaError_t launch_fit_finish(const Batch& b, double* Z, size_t zs, double* scalars, cudaStream_t s) {
    k_fit_finish<<<b.count, kThreads, 0, s>>>(b, Z, zs, scalars);
    return cudaGetLastError();
}

int solve_f64_launches(int nt, bool backward) { return backward ? 2 * nt - 1 : 2 * nt; }

cudaError_t launch_forward_solve(const Batch& b, double* Z, size_t zs, cudaStream_t s) {
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_fwd_diag_f64, kDiagSmem, attr);
    if (e != cudaSuccess) return e;
    const int nt = b.nt;
    k_rhs_f64<<<dim3((nt * GP_NB + kThreads - 1) / kThreads, b.count), kThreads, 0, s>>>(b, Z, zs);
    for (int J = 0; J < nt; ++J) {
        k_fwd_diag_f64<<<b.count, 2 * GP_NB, kDiagSmem, s>>>(b, Z, zs, J);
        if (J + 1 < nt) k_fwd_tiles_f64<<<dim3(nt - 1 - J, b.count), kTileThreads, 0, s>>>(b, Z, zs, J);
    }
    return cudaGetLastError();
}

cudaError_t launch_backward_solve(const Batch& b, double* Z, size_t zs, int col, cudaStream_t s) {
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_bwd_diag_f64, kDiagSmem, attr);
    if (e != cudaSuccess) return e;
    for (int I = b.nt - 1; I >= 0; --I) {
        k_bwd_diag_f64<<<b.count, GP_NB, kDiagSmem, s>>>(b, Z, zs, col, I);
        if (I > 0) k_bwd_tiles_f64<<<dim3(I, b.count), kTileThreads, 0, s>>>(b, Z, zs, col, I);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Batch& b, const double* Z, size_t zs, double* nll, double* mu,
                            double* sigma2, double* logdet, int* status, cudaStream_t s) {
    k_finalize<<<b.count, kThreads, 0, s>>>(b, Z, zs, nll, mu, sigma2, logdet, status);
    return cudaGetLastError();
}

}  // namespace gp
