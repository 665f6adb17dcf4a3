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
// Z[npad..2 npad).  Each instance is solved by one CTA, tile row by tile
// row; reductions run in a fixed order so results do not depend on what
// else is in the batch.
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

// Forward solve of both right-hand sides for one instance per CTA.
__global__ void __launch_bounds__(kThreads) k_forward(Batch b, double* Z, size_t zs) {
    __shared__ double xj[2][GP_NB];
    __shared__ double part[2][2][GP_NB];
    __shared__ double rhs[2][GP_NB];
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    const int nt = b.nt, n = b.n;
    const int npad = nt * GP_NB;
    double* z0 = Z + (size_t)t * zs;
    double* z1 = z0 + npad;
    const int r = threadIdx.x % GP_NB;
    const int h = threadIdx.x / GP_NB;
    for (int I = 0; I < nt; ++I) {
        const int gi = I * GP_NB + r;
        double acc0 = 0.0, acc1 = 0.0;
        for (int Jt = 0; Jt < I; ++Jt) {
            __syncthreads();
            if (h == 0) xj[0][r] = z0[Jt * GP_NB + r];
            else        xj[1][r] = z1[Jt * GP_NB + r];
            __syncthreads();
            const double* L = tile_ptr(b, t, I, Jt);
            // columns c of parity h; thread reads row r of column c (coalesced)
            for (int c = h; c < GP_NB; c += 2) {
                const double l = __ldg(L + c * GP_NB + r);
                acc0 = fma(l, xj[0][c], acc0);
                acc1 = fma(l, xj[1][c], acc1);
            }
        }
        part[h][0][r] = acc0;
        part[h][1][r] = acc1;
        __syncthreads();
        if (h == 0) {
            const double b0 = (gi < n) ? 1.0 : 0.0;
            const double b1 = (gi < n) ? b.y[gi] : 0.0;
            rhs[0][r] = b0 - (part[0][0][r] + part[1][0][r]);
            rhs[1][r] = b1 - (part[0][1][r] + part[1][1][r]);
        }
        __syncthreads();
        // triangular solve with the diagonal tile (lower part holds L_II)
        const double* D = tile_ptr(b, t, I, I);
        for (int c = 0; c < GP_NB; ++c) {
            const double inv = 1.0 / __ldg(D + c * GP_NB + c);
            const double x0 = rhs[0][c] * inv;
            const double x1 = rhs[1][c] * inv;
            __syncthreads();
            if (threadIdx.x < GP_NB && r > c) {
                const double l = __ldg(D + c * GP_NB + r);
                rhs[0][r] = fma(-l, x0, rhs[0][r]);
                rhs[1][r] = fma(-l, x1, rhs[1][r]);
            }
            if (threadIdx.x == 0) { rhs[0][c] = x0; rhs[1][c] = x1; }
            __syncthreads();
        }
        if (h == 0) z0[I * GP_NB + r] = rhs[0][r];
        else        z1[I * GP_NB + r] = rhs[1][r];
        __syncthreads();
    }
}

// Backward solve L^T w = z for column `col` of Z (in place), one CTA per
// instance.  Warp w reduces tile columns w, w+8, ... (coalesced reads).
__global__ void __launch_bounds__(kThreads) k_backward(Batch b, double* Z, size_t zs, int col) {
    __shared__ double wk[GP_NB];
    __shared__ double rhs[GP_NB];
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    const int nt = b.nt;
    const int npad = nt * GP_NB;
    double* z = Z + (size_t)t * zs + (size_t)col * npad;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int I = nt - 1; I >= 0; --I) {
        if (threadIdx.x < GP_NB) rhs[threadIdx.x] = z[I * GP_NB + threadIdx.x];
        __syncthreads();
        for (int K = I + 1; K < nt; ++K) {
            if (threadIdx.x < GP_NB) wk[threadIdx.x] = z[K * GP_NB + threadIdx.x];
            __syncthreads();
            const double* L = tile_ptr(b, t, K, I);   // rows of block K, columns of block I
            for (int c = w; c < GP_NB; c += kThreads / 32) {
                double s = 0.0;
                for (int k = lane; k < GP_NB; k += 32) s = fma(__ldg(L + c * GP_NB + k), wk[k], s);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (lane == 0) rhs[c] -= s;
            }
            __syncthreads();
        }
        const double* D = tile_ptr(b, t, I, I);
        for (int c = GP_NB - 1; c >= 0; --c) {
            const double x = rhs[c] / __ldg(D + c * GP_NB + c);
            __syncthreads();
            if (threadIdx.x < c) rhs[threadIdx.x] = fma(-__ldg(D + threadIdx.x * GP_NB + c), x, rhs[threadIdx.x]);
            if (threadIdx.x == 0) rhs[c] = x;
            __syncthreads();
        }
        if (threadIdx.x < GP_NB) z[I * GP_NB + threadIdx.x] = rhs[threadIdx.x];
        __syncthreads();
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

cudaError_t launch_forward_solve(const Batch& b, double* Z, size_t zs, cudaStream_t s) {
    k_forward<<<b.count, kThreads, 0, s>>>(b, Z, zs);
    return cudaGetLastError();
}

cudaError_t launch_backward_solve(const Batch& b, double* Z, size_t zs, int col, cudaStream_t s) {
    k_backward<<<b.count, kThreads, 0, s>>>(b, Z, zs, col);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Batch& b, const double* Z, size_t zs, double* nll, double* mu,
                            double* sigma2, double* logdet, int* status, cudaStream_t s) {
    k_finalize<<<b.count, kThreads, 0, s>>>(b, Z, zs, nll, mu, sigma2, logdet, status);
    return cudaGetLastError();
}

}  // namespace gp
