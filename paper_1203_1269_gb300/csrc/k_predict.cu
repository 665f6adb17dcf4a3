// k_predict.cu -- kriging mean and variance from a resident fit.
//
// For a test point x*:  r_i = exp(-sum_k theta_k |x*_k - x_ik|^p)  (eq. 2,
// no nugget), yhat = mu_hat + r'w with w = R^-1 (Y - 1 mu_hat), and, with
// v = L^-1 r and a = L^-1 1,
//   s2 = sigma2_hat [c0 - v'v + (1 - a'v)^2 / a'a].
// The paper prices prediction at one R, one factorisation and 2N + 6
// back-solves for N points (Section 3): two triangular solves per point.
//
// The fit is factored in double and its factor, w, a and x are then held as
// double-float pairs (hi + lo floats), so that everything here runs on the
// FP32 pipes: |dx|^p = exp(p ln|dx|) and exp(-S) in double-float arithmetic,
// and the forward solve v = L^-1 r in double-float.
//
// One CTA takes NR test points (16, or 8 when there are too few points to
// give every SM two CTAs at 16) as right-hand sides and walks the tile rows
// of L: it forms the r block of the tile row on the fly, removes the
// solved blocks above it (a 128 x 128 by 128 x 16 product per tile), solves
// with the diagonal tile and folds the finished block into v'v and a'v.
// Solved blocks are kept in a per-CTA slice of `work` (npad x NR pairs).
#include "corr.cuh"
#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;

struct PredArgs {
    int n, d, nt, N, m0;   // m0: first test point of this launch
    const float2* x;       // n x d (double-float)
    const double* theta;   // d
    double p, c0;
    int corr;              // gp_correlation of the fit
    const float2* L;       // packed tiles (double-float)
    const float2* w;       // npad
    const float2* a;       // npad
    const double* sc;      // scalars: nll, mu, sigma2, logdet, Q, aa
    const double* xs;      // N x d
    double* yhat;
    double* s2;
    float2* work;          // per CTA: npad * NR
};

// NR test points per CTA, PT = NR / 2 per thread (two threads per row).
// dynamic shared memory: rhs[NR][NB] + vs[NB][NR] (dfl) + xs[NR][d] + th[d] (dfl) + tab[kExpTab]
template <int NR>
__global__ void __launch_bounds__(kThreads) k_predict(PredArgs g) {
    constexpr int PT = NR / 2;
    extern __shared__ dfl sm[];
    dfl* rhs = sm;                                 // [NR][NB]
    dfl* vs = rhs + NR * GP_NB;                    // [NB][NR]
    dfl* xsm = vs + GP_NB * NR;                    // [NR][d]
    dfl* th = xsm + NR * g.d;                      // [d]
    dfl* tab = th + g.d;                           // [kExpTab]
    __shared__ dfl red[3][NR][4];
    const int d = g.d, n = g.n, nt = g.nt;
    const int npad = nt * GP_NB;
    const int mbase = g.m0 + blockIdx.x * NR;
    const int r = threadIdx.x % GP_NB;
    const int hh = threadIdx.x / GP_NB;            // points hh*PT .. hh*PT+PT-1
    const bool want_var = (g.s2 != nullptr);
    float2* V = g.work + (size_t)blockIdx.x * npad * NR;   // V[i * NR + m]

    for (int q = threadIdx.x; q < NR * d; q += kThreads) {
        const int m = q / d, k = q % d;
        xsm[q] = (mbase + m < g.N) ? df_from_double(g.xs[(size_t)(mbase + m) * d + k]) : dfl{0.f, 0.f};
    }
    // Matern families: theta pre-multiplied by c, powers with p = 1 (corr.cuh)
    for (int q = threadIdx.x; q < d; q += kThreads) th[q] = df_from_double(corr_theta_scale(g.corr) * g.theta[q]);
    fill_exp2_table(tab);
    const dfl pd = df_from_double(g.p);
    const bool matern = corr_is_matern(g.corr);
    const int pmode = matern ? kPowOne : pow_mode(g.p);
    const dfl third = df_from_double(1.0 / 3.0);
    __syncthreads();

    dfl mean_p[PT], vv_p[PT], av_p[PT];
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        mean_p[u] = {0.f, 0.f};
        vv_p[u] = {0.f, 0.f};
        av_p[u] = {0.f, 0.f};
    }

    for (int I = 0; I < nt; ++I) {
        const int gi = I * GP_NB + r;
        const dfl wi = df_load(g.w + gi);
        // r block of this tile row (zero on padded rows)
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            const int m = hh * PT + u;
            dfl v = {0.f, 0.f};
            if (gi < n && mbase + m < g.N) {
                dfl s = {0.f, 0.f}, qp = {1.f, 0.f};
                for (int k = 0; k < d; ++k) {
                    const dfl dx = df_sub(xsm[m * d + k], df_load(g.x + (size_t)gi * d + k));
                    const dfl h = df_mul(th[k], df_powabs(dx, pmode, g.p, pd, tab));
                    s = df_add(s, h);
                    if (matern) qp = df_mul(qp, matern_q_df(h, g.corr, third));
                }
                v = df_exp_neg(s, tab);
                if (matern) v = df_mul(v, qp);
            }
            mean_p[u] = df_fma(v, wi, mean_p[u]);
            rhs[m * GP_NB + r] = v;
        }
        if (!want_var) continue;
        // remove the solved blocks above: rhs -= L_IJ V_J
        dfl acc[PT];
#pragma unroll
        for (int u = 0; u < PT; ++u) acc[u] = {0.f, 0.f};
        for (int J = 0; J < I; ++J) {
            __syncthreads();
            for (int q = threadIdx.x; q < GP_NB * NR; q += kThreads) {
                const float2 v = V[(size_t)J * GP_NB * NR + q];
                vs[q] = dfl{v.x, v.y};
            }
            __syncthreads();
            const float2* Lt = g.L + (size_t)tile_index(I, J, nt) * GP_TILE_ELEMS;
#pragma unroll 2
            for (int c = 0; c < GP_NB; ++c) {
                const float2 lv = __ldg(Lt + c * GP_NB + r);
                const dfl l = {lv.x, lv.y};
#pragma unroll
                for (int u = 0; u < PT; ++u) acc[u] = df_fma(l, vs[c * NR + hh * PT + u], acc[u]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PT; ++u) rhs[(hh * PT + u) * GP_NB + r] = df_sub(rhs[(hh * PT + u) * GP_NB + r], acc[u]);
        __syncthreads();
        // solve with the diagonal tile: thread (r, hh) owns points hh*PT.. of row r
        const float2* D = g.L + (size_t)tile_index(I, I, nt) * GP_TILE_ELEMS;
        for (int c = 0; c < GP_NB; ++c) {
            const float2 dv = __ldg(D + c * GP_NB + c);
            const dfl dc = {dv.x, dv.y};
            dfl lrc = {0.f, 0.f};
            if (r > c) {
                const float2 lv = __ldg(D + c * GP_NB + r);
                lrc = dfl{lv.x, lv.y};
            }
            dfl xc[PT];
#pragma unroll
            for (int u = 0; u < PT; ++u) xc[u] = df_div(rhs[(hh * PT + u) * GP_NB + c], dc);
            __syncthreads();
            if (r > c) {
#pragma unroll
                for (int u = 0; u < PT; ++u)
                    rhs[(hh * PT + u) * GP_NB + r] = df_fms(lrc, xc[u], rhs[(hh * PT + u) * GP_NB + r]);
            } else if (r == c) {
#pragma unroll
                for (int u = 0; u < PT; ++u) rhs[(hh * PT + u) * GP_NB + c] = xc[u];
            }
            __syncthreads();
        }
        const dfl ai = df_load(g.a + gi);
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            const dfl v = rhs[(hh * PT + u) * GP_NB + r];
            V[(size_t)gi * NR + hh * PT + u] = make_float2(v.hi, v.lo);
            vv_p[u] = df_fma(v, v, vv_p[u]);
            av_p[u] = df_fma(ai, v, av_p[u]);
        }
        __syncthreads();
    }
    // reduce over the 128 rows for each point: warp shuffles, then 4 warps
    const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 3;
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        dfl t3[3] = {mean_p[u], vv_p[u], av_p[u]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            for (int o = 16; o > 0; o >>= 1) {
                dfl w2;
                w2.hi = __shfl_down_sync(0xffffffffu, t3[k].hi, o);
                w2.lo = __shfl_down_sync(0xffffffffu, t3[k].lo, o);
                t3[k] = df_add(t3[k], w2);
            }
            if (lane == 0) red[k][hh * PT + u][wq] = t3[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        const int m = threadIdx.x;
        if (mbase + m < g.N) {
            const double mu = g.sc[1], sigma2 = g.sc[2], aa = g.sc[5];
            dfl s3[3];
            for (int k = 0; k < 3; ++k)
                s3[k] = df_add(df_add(red[k][m][0], red[k][m][1]), df_add(red[k][m][2], red[k][m][3]));
            g.yhat[mbase + m] = mu + df_to_double(s3[0]);
            if (want_var) {
                const double vv = df_to_double(s3[1]);
                const double gg = 1.0 - df_to_double(s3[2]);
                g.s2[mbase + m] = sigma2 * (g.c0 - vv + gg * gg / aa);
            }
        }
    }
}

// In-place double -> double-float conversion of a fitted model's arrays.
__global__ void k_to_df_inplace(double* p, size_t count) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const double v = p[i];
        const float h = __double2float_rn(v);
        const float l = __double2float_rn(v - (double)h);
        reinterpret_cast<float2*>(p)[i] = make_float2(h, l);
    }
}

}  // namespace

cudaError_t launch_to_df_inplace(double* p, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_to_df_inplace<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, count);
    return cudaGetLastError();
}

size_t predict_work_per_cta(int nt, int nr) { return (size_t)nt * GP_NB * nr * sizeof(float2); }

int predict_points_per_cta(int N, int sms) { return (N + 15) / 16 < 2 * sms ? 8 : 16; }

template <int NR>
static cudaError_t launch_predict_nr(const PredArgs& g0, int d, int N, int chunk, cudaStream_t s) {
    const size_t smem = (size_t)(2 * NR * GP_NB + NR * d + d + kExpTab) * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_predict<NR>, smem, attr);
    if (e != cudaSuccess) return e;
    PredArgs g = g0;
    const int blocks_total = (N + NR - 1) / NR;
    for (int b0 = 0; b0 < blocks_total; b0 += chunk) {
        const int nb = (blocks_total - b0 < chunk) ? (blocks_total - b0) : chunk;
        g.m0 = b0 * NR;
        k_predict<NR><<<nb, kThreads, smem, s>>>(g);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_predict(int n, int d, int nt, const float2* x, const double* theta, double p, int corr, double c0,
                           const float2* L, const float2* w, const float2* a, const double* scalars, int N,
                           const double* xs, double* yhat, double* s2, float2* work, int chunk, int nr,
                           cudaStream_t s) {
    PredArgs g;
    g.n = n; g.d = d; g.nt = nt; g.N = N; g.m0 = 0;
    g.x = x; g.theta = theta; g.p = p; g.corr = corr; g.c0 = c0;
    g.L = L; g.w = w; g.a = a; g.sc = scalars; g.xs = xs; g.yhat = yhat; g.s2 = s2; g.work = work;
    if (nr == 8) return launch_predict_nr<8>(g, d, N, chunk, s);
    if (nr == 16) return launch_predict_nr<16>(g, d, N, chunk, s);
    return cudaErrorInvalidValue;
}

}  // namespace gp
