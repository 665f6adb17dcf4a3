// k_predict.cu -- kriging mean and variance from a resident fit.
//
// For a test point x*:  r_i = prod_k exp(-theta_k |x*_k - x_ik|^p)  (eq. 2,
// no nugget), yhat = mu_hat + r'w with w = R^-1 (Y - 1 mu_hat), and, with
// v = L^-1 r and a = L^-1 1,
//   s2 = sigma2_hat [c0 - v'v + (1 - a'v)^2 / a'a].
// The paper prices prediction at one R, one factorisation and 2N + 6
// back-solves for N points (Section 3): two triangular solves per point.
//
// One CTA takes NR = 32 test points as right-hand sides and walks the tile
// rows of L: it forms the r block of the tile row on the fly, removes the
// solved blocks above it (a 128 x 128 by 128 x 32 product per tile), solves
// with the diagonal tile and folds the finished block into v'v and a'v.
// Solved blocks are kept in a per-CTA slice of `work` (npad x NR doubles).
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;
constexpr int NR = 32;

__device__ __forceinline__ double powabs_p(double diff, double p) {
    double a = fabs(diff);
    if (p == 2.0) return a * a;
    if (p == 1.0) return a;
    return (a == 0.0) ? 0.0 : pow(a, p);
}

struct PredArgs {
    int n, d, nt, N, m0;   // m0: first test point of this launch
    const double* x;       // n x d
    const double* theta;   // d
    double p, c0;
    const double* L;       // packed tiles
    const double* w;       // npad
    const double* a;       // npad
    const double* sc;      // scalars: nll, mu, sigma2, logdet, Q, aa
    const double* xs;      // N x d
    double* yhat;
    double* s2;
    double* work;          // per CTA: npad * NR
};

// dynamic shared memory: rhs[NR][NB] + vs[NB][NR] + xs[NR][d] + th[d]
__global__ void __launch_bounds__(kThreads) k_predict(PredArgs g) {
    extern __shared__ double sm[];
    double* rhs = sm;                              // [NR][NB]
    double* vs = rhs + NR * GP_NB;                 // [NB][NR]
    double* xsm = vs + GP_NB * NR;                 // [NR][d]
    double* th = xsm + NR * g.d;                   // [d]
    __shared__ double red[2][NR][4];
    const int d = g.d, n = g.n, nt = g.nt;
    const int npad = nt * GP_NB;
    const int mbase = g.m0 + blockIdx.x * NR;
    const int r = threadIdx.x % GP_NB;
    const int hh = threadIdx.x / GP_NB;           // 0..1 -> points hh*16 .. hh*16+15
    const bool want_var = (g.s2 != nullptr);
    double* V = g.work + (size_t)blockIdx.x * npad * NR;   // V[i * NR + m]

    for (int q = threadIdx.x; q < NR * d; q += kThreads) {
        const int m = q / d, k = q % d;
        xsm[q] = (mbase + m < g.N) ? g.xs[(size_t)(mbase + m) * d + k] : 0.0;
    }
    for (int q = threadIdx.x; q < d; q += kThreads) th[q] = g.theta[q];
    __syncthreads();

    double mean_p[16], vv_p[16], av_p[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) { mean_p[u] = 0.0; vv_p[u] = 0.0; av_p[u] = 0.0; }

    for (int I = 0; I < nt; ++I) {
        const int gi = I * GP_NB + r;
        const double wi = g.w[gi];
        // r block of this tile row (zero on padded rows)
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int m = hh * 16 + u;
            double v = 0.0;
            if (gi < n && mbase + m < g.N) {
                double s = 0.0;
                for (int k = 0; k < d; ++k)
                    s = fma(th[k], powabs_p(xsm[m * d + k] - g.x[(size_t)gi * d + k], g.p), s);
                v = exp(-s);
            }
            mean_p[u] = fma(v, wi, mean_p[u]);
            rhs[m * GP_NB + r] = v;
        }
        if (!want_var) continue;
        // remove the solved blocks above: rhs -= L_IJ V_J
        double acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.0;
        for (int J = 0; J < I; ++J) {
            __syncthreads();
            for (int q = threadIdx.x; q < GP_NB * NR; q += kThreads) vs[q] = V[(size_t)J * GP_NB * NR + q];
            __syncthreads();
            const double* Lt = g.L + (size_t)tile_index(I, J, nt) * GP_TILE_ELEMS;
            for (int c = 0; c < GP_NB; ++c) {
                const double l = __ldg(Lt + c * GP_NB + r);
#pragma unroll
                for (int u = 0; u < 16; ++u) acc[u] = fma(l, vs[c * NR + hh * 16 + u], acc[u]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; ++u) rhs[(hh * 16 + u) * GP_NB + r] -= acc[u];
        __syncthreads();
        // solve with the diagonal tile: thread (r, hh) owns points hh*16..+15 of row r
        const double* D = g.L + (size_t)tile_index(I, I, nt) * GP_TILE_ELEMS;
        for (int c = 0; c < GP_NB; ++c) {
            const double inv = 1.0 / __ldg(D + c * GP_NB + c);
            const double lrc = (r > c) ? __ldg(D + c * GP_NB + r) : 0.0;
            double xc[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) xc[u] = rhs[(hh * 16 + u) * GP_NB + c] * inv;
            __syncthreads();
            if (r > c) {
#pragma unroll
                for (int u = 0; u < 16; ++u) rhs[(hh * 16 + u) * GP_NB + r] = fma(-lrc, xc[u], rhs[(hh * 16 + u) * GP_NB + r]);
            } else if (r == c) {
#pragma unroll
                for (int u = 0; u < 16; ++u) rhs[(hh * 16 + u) * GP_NB + c] = xc[u];
            }
            __syncthreads();
        }
        const double ai = g.a[gi];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const double v = rhs[(hh * 16 + u) * GP_NB + r];
            V[(size_t)gi * NR + hh * 16 + u] = v;
            vv_p[u] = fma(v, v, vv_p[u]);
            av_p[u] = fma(ai, v, av_p[u]);
        }
        __syncthreads();
    }
    // reduce over the 128 rows for each point: warp shuffles then 4 warps
    const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 3;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        double m1 = mean_p[u], m2 = vv_p[u], m3 = av_p[u];
        for (int o = 16; o > 0; o >>= 1) {
            m1 += __shfl_down_sync(0xffffffffu, m1, o);
            m2 += __shfl_down_sync(0xffffffffu, m2, o);
            m3 += __shfl_down_sync(0xffffffffu, m3, o);
        }
        if (lane == 0) {
            red[0][hh * 16 + u][wq] = m1;
            red[1][hh * 16 + u][wq] = m2;
            // a'v partials reuse rhs (free now) to keep `red` small
            rhs[(hh * 16 + u) * 4 + wq] = m3;
        }
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        const int m = threadIdx.x;
        if (mbase + m < g.N) {
            const double mu = g.sc[1], sigma2 = g.sc[2], aa = g.sc[5];
            const double mean = red[0][m][0] + red[0][m][1] + red[0][m][2] + red[0][m][3];
            g.yhat[mbase + m] = mu + mean;
            if (want_var) {
                const double vv = red[1][m][0] + red[1][m][1] + red[1][m][2] + red[1][m][3];
                const double av = rhs[m * 4 + 0] + rhs[m * 4 + 1] + rhs[m * 4 + 2] + rhs[m * 4 + 3];
                const double gg = 1.0 - av;
                g.s2[mbase + m] = sigma2 * (g.c0 - vv + gg * gg / aa);
            }
        }
    }
}

}  // namespace

cudaError_t launch_predict(int n, int d, int nt, const double* x, const double* theta, double p,
                           double c0, const double* L, const double* w, const double* a,
                           const double* scalars, int N, const double* xs, double* yhat,
                           double* s2, double* work, int chunk, cudaStream_t s) {
    const size_t smem = (size_t)(2 * NR * GP_NB + NR * d + d) * sizeof(double);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    PredArgs g;
    g.n = n; g.d = d; g.nt = nt; g.N = N;
    g.x = x; g.theta = theta; g.p = p; g.c0 = c0;
    g.L = L; g.w = w; g.a = a; g.sc = scalars; g.xs = xs; g.yhat = yhat; g.s2 = s2; g.work = work;
    const int blocks_total = (N + NR - 1) / NR;
    for (int b0 = 0; b0 < blocks_total; b0 += chunk) {
        const int nb = (blocks_total - b0 < chunk) ? (blocks_total - b0) : chunk;
        g.m0 = b0 * NR;
        k_predict<<<nb, kThreads, smem, s>>>(g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gp
