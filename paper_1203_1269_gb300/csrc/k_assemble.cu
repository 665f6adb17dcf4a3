// k_assemble.cu -- the power-exponential correlation matrix (Section 2,
// eq. 2) with a diagonal nugget, written straight into the factorisation's
// tile storage for a batch of theta candidates.
//
// R_ij = exp(-sum_k theta_k |x_ik - x_jk|^p) + delta [i == j]
//
// The d powers |x_ik - x_jk|^p do not depend on theta, so each thread
// computes them once per matrix entry and reuses them for every candidate of
// its group; per candidate an entry then costs d FMAs and one exp.  The paper
// counts d n(n-1)/2 independent terms (Section 3); here the lower triangle of
// tiles (diagonal tiles in full) is produced.
//
// The double-float variant (split-precision path) keeps everything on the
// FP32 pipes: on this GPU one FP64 pow costs as much as thousands of FP32
// instructions, so the powers are exp(p ln|dx|) in double-float too.
#include <cmath>

#include "corr.cuh"
#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 256;
constexpr int kSplit = 4;                       // a CTA covers NB/kSplit columns of a tile
constexpr int kCols = GP_NB / kSplit;           // 32 columns
constexpr int kEntries = GP_NB * kCols / kThreads;  // 16 entries per thread
// double-float variant: COLS (16 or 32) tile columns per CTA -- narrower
// parts fill the last wave of CTAs better, wider ones share each theta
// load over more entries

__device__ __forceinline__ double powabs(double diff, double p) {
    double a = fabs(diff);
    if (p == 2.0) return a * a;
    if (p == 1.0) return a;
    return (a == 0.0) ? 0.0 : pow(a, p);
}

// |dx|^p in double for a general p without a pow per term (the reduction
// of P. T. P. Tang's table-driven logarithm, ACM TOMS 16 (1990), applied to
// the power): a = 2^m F_j (1 + u) with F_j = 1 + j/64 the table point
// nearest the mantissa (|u| <= 2^-7), so that
//   a^p = [2^(m p) F_j^p] (1 + u)^p,
// the bracket as a double-double product of two tables computed on the host
// in long double, (1 + u)^p - 1 = p u + c2 u^2 + ... + c7 u^7 (the u^8 term
// is below 2^-62), and one rounding at the end: a^p = A_hi + (A_hi t +
// A_lo).  m outside [-60, 4] takes pow.
constexpr int kP64NBits = 6;
constexpr int kP64N = 1 << kP64NBits;
constexpr int kP64Mlo = -60, kP64Mhi = 4;
constexpr int kP64Ms = kP64Mhi - kP64Mlo + 1;
struct PowTab64 {
    int on;                       // general p on the power-exponential family
    double c[8];                  // c[k] = C(p, k), k = 1 .. 7
    double inv[kP64N];            // 1 / F_j (rounded: the division's residual is formed exactly)
    double2 two[kP64Ms];          // 2^(m p), m = kP64Mlo .. kP64Mhi, as (hi, lo)
    double2 f[kP64N];             // F_j^p as (hi, lo)
};
static_assert(sizeof(PowTab64) + 512 < 4096, "kernel parameters");

__device__ __forceinline__ double pow_tab64(double a, double p, const PowTab64& t) {
    const long long rb = __double_as_longlong(a) + (1LL << (51 - kP64NBits));   // a > 0
    const int e = (int)(rb >> 52);
    if (e - 1023 < kP64Mlo || e - 1023 > kP64Mhi) return pow(a, p);
    const int j = (int)(rb >> (52 - kP64NBits)) & (kP64N - 1);
    const double Fm = __longlong_as_double(rb & ~((1LL << (52 - kP64NBits)) - 1));   // 2^m F_j
    const double g = __longlong_as_double((long long)(2046 - e) << 52);              // 2^-m
    const double fh = (a - Fm) * g;                                                   // exact
    const double F = Fm * g;
    const double iv = t.inv[j];
    const double uh = fh * iv;
    const double ul = fma(-uh, F, fh) * iv;
    double q = fma(uh, t.c[7], t.c[6]);
    q = fma(uh, q, t.c[5]);
    q = fma(uh, q, t.c[4]);
    q = fma(uh, q, t.c[3]);
    q = fma(uh, q, t.c[2]);
    const double tt = fma(t.c[1], uh, fma(t.c[1], ul, uh * uh * q));
    const double2 T = t.two[e - 1023 - kP64Mlo], P = t.f[j];
    const double ah = T.x * P.x;
    const double al = fma(T.x, P.x, -ah) + fma(T.x, P.y, T.y * P.x);
    return ah + fma(ah, tt, al);
}

__device__ __forceinline__ double powabs_t(double diff, double p, const PowTab64& t) {
    const double a = fabs(diff);
    return (a == 0.0) ? 0.0 : pow_tab64(a, p, t);
}

// |dx|^p as double-float: p = 2 and p = 1 exactly in double (one FP64
// multiply), any other p as exp(p ln|dx|) in double-float arithmetic.
// Values are clamped to 2^120 so that the float range holds them.
__device__ __forceinline__ dfl power_term(double dx, int pmode, double p, dfl pd, const dfl* tab) {
    if (pmode == kPowTwo) return df_from_double(fmin(dx * dx, 0x1p120));
    if (pmode == kPowOne) return df_from_double(fmin(fabs(dx), 0x1p120));
    return df_powabs(df_from_double(dx), kPowGeneral, p, pd, tab);
}

// One entry of instance t: double tiles, or double-float working matrix plus
// its double-float copy (split-precision path).
__device__ __forceinline__ void store_entry(const Batch& b, int t, size_t off, double v) {
    const size_t i = (size_t)t * b.inst_stride + off;
    if (b.Adf) {
        const float h = __double2float_rn(v);
        const float l = __double2float_rn(v - (double)h);
        const float2 hl = make_float2(h, l);
        b.Adf[i] = hl;
        b.Rdf[i] = hl;
    } else {
        b.A[i] = v;
    }
}

// Validate theta and reset each instance's record.
__global__ void k_validate_theta(Batch b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.count) return;
    int bad = 0;
    for (int k = 0; k < b.d; ++k) {
        double th = b.theta[(size_t)t * b.d + k];
        if (!(th >= 0.0) || !isfinite(th)) bad = 1;
    }
    InstState s;
    s.logdet = 0.0; s.aa = 0.0; s.ab = 0.0; s.mu = 0.0; s.Q = 0.0; s.bb = 0.0;
    s.status = bad ? GP_EINVAL : GP_OK;
    s.fail_col = -1;
    s.anorm = 0.0; s.est = 0.0;
    s.hager_iter = 0; s.hager_jprev = -1; s.hager_done = 0;
    s.piv_inv = 0.0; s.dq_prev = 0.0; s.refine_done = 0;
    b.st[t] = s;
}

// grid.x = packed tiles * kSplit, grid.y = candidate groups; DB = bound on d;
// TAB: a general p on the power-exponential family, powers by pow_tab64
template <int DB, bool TAB>
__global__ void __launch_bounds__(kThreads)
k_assemble_tiles(Batch b, int group, PowTab64 ptab) {
    __shared__ double xs_r[GP_NB * DB];
    __shared__ double xs_c[kCols * DB];
    __shared__ PowTab64 pt;
    if (TAB)
        for (int q = threadIdx.x; q < (int)(sizeof(PowTab64) / sizeof(int)); q += kThreads)
            reinterpret_cast<int*>(&pt)[q] = reinterpret_cast<const int*>(&ptab)[q];
    const int nt = b.nt, n = b.n, d = b.d;
    const int tile_lin = blockIdx.x / kSplit;
    const int part = blockIdx.x % kSplit;
    // decode packed tile index -> (I, J) with column-major tile packing
    int J = 0;
    {
        long long rem = tile_lin;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
        // I = J + rem
        (void)rem;
    }
    long long start = tile_index(J, J, nt);
    const int I = J + (int)(tile_lin - start);
    const int row0 = I * GP_NB, col0 = J * GP_NB + part * kCols;

    for (int q = threadIdx.x; q < GP_NB * DB; q += kThreads) {
        int r = q / DB, k = q % DB;
        int gi = row0 + r;
        xs_r[q] = (gi < n && k < d) ? b.x[(size_t)gi * d + k] : 0.0;
    }
    for (int q = threadIdx.x; q < kCols * DB; q += kThreads) {
        int c = q / DB, k = q % DB;
        int gj = col0 + c;
        xs_c[q] = (gj < n && k < d) ? b.x[(size_t)gj * d + k] : 0.0;
    }
    __syncthreads();

    const int t0 = blockIdx.y * group;
    const int t1 = min(b.count, t0 + group);
    const size_t tile_off = (size_t)tile_lin * GP_TILE_ELEMS;
    const int r = threadIdx.x % GP_NB;           // row inside the tile
    const int cb = threadIdx.x / GP_NB;          // 0..1
    const int gi = row0 + r;
    const bool matern = corr_is_matern(b.corr);
    const double cm = corr_theta_scale(b.corr);

#pragma unroll 1
    for (int e = 0; e < kEntries; ++e) {
        const int c = cb + 2 * e;                // column inside this part
        const int gj = col0 + c;
        const size_t off = tile_off + (size_t)(part * kCols + c) * GP_NB + r;
        const bool pad = (gi >= n) || (gj >= n);
        const bool diag = (gi == gj);
        double D[DB];
#pragma unroll
        for (int k = 0; k < DB; ++k)
            D[k] = (k < d && !pad) ? (matern ? fabs(xs_r[r * DB + k] - xs_c[c * DB + k])
                                             : (TAB ? powabs_t(xs_r[r * DB + k] - xs_c[c * DB + k], b.p, pt)
                                                    : powabs(xs_r[r * DB + k] - xs_c[c * DB + k], b.p)))
                                   : 0.0;
#pragma unroll 1
        for (int t = t0; t < t1; ++t) {
            if (b.st[t].status != GP_OK) continue;
            double v;
            if (pad) {
                v = diag ? 1.0 : 0.0;
            } else {
                const double* th = b.theta + (size_t)t * d;
                double s = 0.0, q = 1.0;
#pragma unroll
                for (int k = 0; k < DB; ++k) {
                    if (k < d) {
                        const double h = cm * __ldg(th + k) * D[k];
                        s += h;
                        if (matern) q *= matern_q(h, b.corr);
                    }
                }
                v = q * exp(-s);
                if (diag) v += b.delta;
            }
            store_entry(b, t, off, v);
        }
    }
}

// Double-float variant for the split-precision path: the powers once per
// entry, then per candidate S = sum_k theta_k D_k and exp(-S), all in
// double-float arithmetic on the FP32 pipes.  Every term of S is >= 0, so S
// is summed with one TwoSum per term on the high parts, the rounding errors
// of the products and the cross terms gathered in one float and folded in at
// the end (about 2^-46 relative, the accuracy of a double-float FMA chain at
// two thirds of its instructions).  Writes the working matrix and its copy.
// Dynamic smem: x rows/cols (double), theta of the group and the exp table
// (double-float), the group's status flags.
// EXACT: DB is d itself, so the loops over the dimensions have a constant
// bound (the benchmark's d = 6: 10.84 -> 9.92 ms, the same bits).
template <int DB, int COLS, bool MATERN, bool EXACT = false>
__global__ void __launch_bounds__(kThreads)
k_assemble_tiles_df(Batch b, int group) {
    constexpr int kSplitDf = GP_NB / COLS;
    constexpr int kColsDf = COLS;
    constexpr int kEntriesDf = GP_NB * COLS / kThreads;
    extern __shared__ double dsm[];
    double* xs_r = dsm;                                  // GP_NB * DB
    double* xs_c = xs_r + GP_NB * DB;                    // kColsDf * DB
    dfl* th = reinterpret_cast<dfl*>(xs_c + kColsDf * DB); // group * DB
    dfl* tab = th + (size_t)group * DB;                  // kExpTab
    int* live = reinterpret_cast<int*>(tab + kExpTab);   // group
    const int nt = b.nt, n = b.n, d = b.d;
    const int tile_lin = blockIdx.x / kSplitDf;
    const int part = blockIdx.x % kSplitDf;
    int J = 0;
    {
        long long rem = tile_lin;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(tile_lin - tile_index(J, J, nt));
    const int row0 = I * GP_NB, col0 = J * GP_NB + part * kColsDf;
    const int t0 = blockIdx.y * group;
    const int t1 = min(b.count, t0 + group);
    for (int q = threadIdx.x; q < GP_NB * DB; q += kThreads) {
        const int r = q / DB, k = q % DB, gi = row0 + r;
        xs_r[q] = (gi < n && k < d) ? b.x[(size_t)gi * d + k] : 0.0;
    }
    for (int q = threadIdx.x; q < kColsDf * DB; q += kThreads) {
        const int c = q / DB, k = q % DB, gj = col0 + c;
        xs_c[q] = (gj < n && k < d) ? b.x[(size_t)gj * d + k] : 0.0;
    }
    for (int q = threadIdx.x; q < (t1 - t0) * DB; q += kThreads) {
        const int tt = q / DB, k = q % DB;
        th[q] = (k < d) ? df_from_double(corr_theta_scale(b.corr) * b.theta[(size_t)(t0 + tt) * d + k])
                        : dfl{0.f, 0.f};
    }
    for (int q = threadIdx.x; q < t1 - t0; q += kThreads) live[q] = (b.st[t0 + q].status == GP_OK);
    fill_exp2_table(tab);
    __syncthreads();
    const dfl delta = df_from_double(b.delta);
    constexpr bool matern = MATERN;                          // the family is a template argument
    const int pmode = matern ? kPowOne : pow_mode(b.p);      // Matern: h = c theta |dx|
    const dfl pd = df_from_double(b.p);
    const dfl third = df_from_double(1.0 / 3.0);
    const size_t tile_off = (size_t)tile_lin * GP_TILE_ELEMS;
    const int r = threadIdx.x % GP_NB;
    const int cb = threadIdx.x / GP_NB;
    const int gi = row0 + r;
#pragma unroll 1
    for (int e = 0; e < kEntriesDf; ++e) {
        const int c = cb + 2 * e;
        const int gj = col0 + c;
        const size_t off = tile_off + (size_t)(part * kColsDf + c) * GP_NB + r;
        const bool pad = (gi >= n) || (gj >= n);
        const bool diag = (gi == gj);
        dfl D[DB];
#pragma unroll
        for (int k = 0; k < DB; ++k)
            D[k] = (k < (EXACT ? DB : d) && !pad) ? power_term(xs_r[r * DB + k] - xs_c[c * DB + k], pmode, b.p, pd, tab)
                                   : dfl{0.f, 0.f};
#pragma unroll 1
        for (int t = t0; t < t1; ++t) {
            if (!live[t - t0]) continue;
            dfl v;
            if (pad) {
                v = {diag ? 1.f : 0.f, 0.f};
            } else {
                const dfl* tt = th + (size_t)(t - t0) * DB;
                float sh = 0.f, sl = 0.f;
                dfl qp = {1.f, 0.f};                // Matern: prod_k q(h_k)
                // k >= d is uniform across the warp: leave the unrolled loop
                // there rather than issue its predicated-off iterations; the
                // first term enters S exactly (the TwoSum of 0 and it is exact)
#pragma unroll
                for (int k = 0; k < DB; ++k) {
                    if (k >= (EXACT ? DB : d)) break;
                    const dfl a = tt[k];
                    float ph = __fmul_rn(a.hi, D[k].hi);
                    if (matern) {
                        // h_k = a D_k itself is needed for q(h_k): its high
                        // word enters the TwoSum, its low word sl
                        const float pe = __fmaf_rn(a.hi, D[k].hi, -ph);
                        const float pl = __fmaf_rn(a.hi, D[k].lo, __fmul_rn(a.lo, D[k].hi));
                        dfl h;
                        fast_two_sum(ph, __fadd_rn(pe, pl), h.hi, h.lo);
                        qp = df_mul(qp, matern_q_df(h, b.corr, third));
                        ph = h.hi;
                        sl = __fadd_rn(sl, h.lo);
                    } else {
                        sl = __fadd_rn(sl, __fmaf_rn(a.hi, D[k].hi, -ph));
                        sl = __fmaf_rn(a.hi, D[k].lo, sl);
                        sl = __fmaf_rn(a.lo, D[k].hi, sl);
                    }
                    if (k == 0) {
                        sh = ph;
                    } else {
                        float s2, e2;
                        two_sum(sh, ph, s2, e2);
                        sh = s2;
                        sl = __fadd_rn(sl, e2);
                    }
                }
                dfl S;
                fast_two_sum(sh, sl, S.hi, S.lo);   // |sl| << sh: every term is >= 0
                v = df_exp_neg(S, tab);
                if (matern) v = df_mul(v, qp);
                if (diag) v = df_add(v, delta);
            }
            const size_t i = (size_t)t * b.inst_stride + off;
            const float2 hl = make_float2(v.hi, v.lo);
            b.Adf[i] = hl;
            b.Rdf[i] = hl;
        }
    }
}

// d above the register-bounded variants: recompute the powers per candidate.
__global__ void __launch_bounds__(kThreads)
k_assemble_tiles_generic(Batch b, int group) {
    const int nt = b.nt, n = b.n, d = b.d;
    const int tile_lin = blockIdx.x / kSplit;
    const int part = blockIdx.x % kSplit;
    int J = 0;
    {
        long long rem = tile_lin;
        while (rem >= nt - J) { rem -= nt - J; ++J; }
    }
    const int I = J + (int)(tile_lin - tile_index(J, J, nt));
    const int row0 = I * GP_NB, col0 = J * GP_NB + part * kCols;
    const int t0 = blockIdx.y * group;
    const int t1 = min(b.count, t0 + group);
    const size_t tile_off = (size_t)tile_lin * GP_TILE_ELEMS;
    const int r = threadIdx.x % GP_NB;
    const int cb = threadIdx.x / GP_NB;
    const int gi = row0 + r;
    for (int e = 0; e < kEntries; ++e) {
        const int c = cb + 2 * e;
        const int gj = col0 + c;
        const size_t off = tile_off + (size_t)(part * kCols + c) * GP_NB + r;
        const bool pad = (gi >= n) || (gj >= n);
        const bool diag = (gi == gj);
        for (int t = t0; t < t1; ++t) {
            if (b.st[t].status != GP_OK) continue;
            double v;
            if (pad) {
                v = diag ? 1.0 : 0.0;
            } else {
                const double* th = b.theta + (size_t)t * d;
                const bool matern = corr_is_matern(b.corr);
                const double cm = corr_theta_scale(b.corr);
                double s = 0.0, q = 1.0;
                for (int k = 0; k < d; ++k) {
                    const double dx = b.x[(size_t)gi * d + k] - b.x[(size_t)gj * d + k];
                    const double h = cm * th[k] * (matern ? fabs(dx) : powabs(dx, b.p));
                    s += h;
                    if (matern) q *= matern_q(h, b.corr);
                }
                v = q * exp(-s);
                if (diag) v += b.delta;
            }
            store_entry(b, t, off, v);
        }
    }
}

// Dense n x n row-major R (both triangles) for one theta.
__global__ void k_assemble_dense(int n, int d, const double* __restrict__ x,
                                 const double* __restrict__ theta, double p, int corr, double delta,
                                 double* __restrict__ R) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n) return;
    const bool matern = corr_is_matern(corr);
    const double cm = corr_theta_scale(corr);
    double s = 0.0, q = 1.0;
    for (int k = 0; k < d; ++k) {
        const double dx = x[(size_t)i * d + k] - x[(size_t)j * d + k];
        const double h = cm * theta[k] * (matern ? fabs(dx) : powabs(dx, p));
        s += h;
        if (matern) q *= matern_q(h, corr);
    }
    double v = q * exp(-s);
    if (i == j) v += delta;
    R[(size_t)i * n + j] = v;
}

}  // namespace

// The double-float assembly for one (DB, COLS, family): its shared-memory
// limit raised once per device and size (raise_smem_limit, safe when
// contexts on several threads assemble at once), then the launch.
template <int DB, int COLS, bool M, bool EXACT = false>
static cudaError_t launch_asm_df(dim3 grid, size_t smem, cudaStream_t s, const Batch& b, int group) {
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_assemble_tiles_df<DB, COLS, M, EXACT>, smem, attr);
    if (e != cudaSuccess) return e;
    k_assemble_tiles_df<DB, COLS, M, EXACT><<<grid, kThreads, smem, s>>>(b, group);
    return cudaGetLastError();
}

// The tables of pow_tab64 for p, in long double (64 significant bits or
// more), rounded to double-double; the last p's tables are kept per thread.
static void pow_tab64_fill(double p, PowTab64& t) {
    static thread_local double last_p = -1.0;
    static thread_local PowTab64 last{};
    if (p != last_p) {
        last = PowTab64{};
        last.on = 1;
        long double c = 1.0L;
        for (int k = 1; k < 8; ++k) {
            c = c * ((long double)p - (long double)(k - 1)) / (long double)k;
            last.c[k] = (double)c;
        }
        last.c[0] = 1.0;
        auto split = [](long double v) {
            const double h = (double)v;
            return make_double2(h, (double)(v - (long double)h));
        };
        for (int j = 0; j < kP64N; ++j) {
            const long double F = 1.0L + (long double)j / (long double)kP64N;
            last.inv[j] = (double)(1.0L / F);
            last.f[j] = split(powl(F, (long double)p));
        }
        for (int m = kP64Mlo; m <= kP64Mhi; ++m) last.two[m - kP64Mlo] = split(exp2l((long double)m * (long double)p));
        last_p = p;
    }
    t = last;
}

cudaError_t launch_validate_theta(const Batch& b, cudaStream_t s) {
    k_validate_theta<<<(b.count + 127) / 128, 128, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_assemble_tiles(const Batch& b, cudaStream_t s) {
    const long long tiles = packed_tiles(b.nt);
    const long long ctas_per_group = tiles * kSplit;
    // enough candidate groups to give ~4 CTAs per SM, but as few as possible
    // so that the theta-independent powers are shared by many candidates
    long long groups = (4 * 152 + ctas_per_group - 1) / ctas_per_group;
    if (groups < 1) groups = 1;
    if (groups > b.count) groups = b.count;
    int group = (int)((b.count + groups - 1) / groups);
    groups = (b.count + group - 1) / group;
    dim3 grid((unsigned)ctas_per_group, (unsigned)groups);
    if (b.Adf && b.d <= 16) {
        const int cols = (b.asm_cols == 32) ? 32 : 16;
        const int split = GP_NB / cols;
        long long g_df = (4 * 152 + tiles * split - 1) / (tiles * split);
        if (g_df < 1) g_df = 1;
        if (g_df > b.count) g_df = b.count;
        group = (int)((b.count + g_df - 1) / g_df);
        g_df = (b.count + group - 1) / group;
        grid = dim3((unsigned)(tiles * split), (unsigned)g_df);
        // 16 columns (the default): DB = d exactly; 32: d rounded up to 4, 8 or 16
        const int DB = (cols == 16) ? b.d : (b.d <= 4 ? 4 : (b.d <= 8 ? 8 : 16));
        const size_t smem = (size_t)(GP_NB + cols) * DB * sizeof(double) +
                            ((size_t)group * DB + kExpTab) * sizeof(dfl) + (size_t)group * sizeof(int);
        const bool m = corr_is_matern(b.corr);
        cudaError_t e;
        if (cols == 16) {
#define GP_ASM_EXACT(D)                                                                                  \
    case D:                                                                                              \
        e = m ? launch_asm_df<D, 16, true, true>(grid, smem, s, b, group)                                \
              : launch_asm_df<D, 16, false, true>(grid, smem, s, b, group);                             \
        break
            switch (b.d) {
                GP_ASM_EXACT(1); GP_ASM_EXACT(2); GP_ASM_EXACT(3); GP_ASM_EXACT(4);
                GP_ASM_EXACT(5); GP_ASM_EXACT(6); GP_ASM_EXACT(7); GP_ASM_EXACT(8);
                GP_ASM_EXACT(9); GP_ASM_EXACT(10); GP_ASM_EXACT(11); GP_ASM_EXACT(12);
                GP_ASM_EXACT(13); GP_ASM_EXACT(14); GP_ASM_EXACT(15); GP_ASM_EXACT(16);
                default: e = cudaErrorInvalidValue;
            }
#undef GP_ASM_EXACT
        } else {
            if (DB == 4) e = m ? launch_asm_df<4, 32, true>(grid, smem, s, b, group) : launch_asm_df<4, 32, false>(grid, smem, s, b, group);
            else if (DB == 8) e = m ? launch_asm_df<8, 32, true>(grid, smem, s, b, group) : launch_asm_df<8, 32, false>(grid, smem, s, b, group);
            else e = m ? launch_asm_df<16, 32, true>(grid, smem, s, b, group) : launch_asm_df<16, 32, false>(grid, smem, s, b, group);
        }
        return e;
    }
    PowTab64 pt{};
    if (b.d <= 16 && !corr_is_matern(b.corr) && pow_mode(b.p) == kPowGeneral) pow_tab64_fill(b.p, pt);
    const bool tab = pt.on != 0;
    if (b.d <= 4)
        tab ? k_assemble_tiles<4, true><<<grid, kThreads, 0, s>>>(b, group, pt)
            : k_assemble_tiles<4, false><<<grid, kThreads, 0, s>>>(b, group, pt);
    else if (b.d <= 8)
        tab ? k_assemble_tiles<8, true><<<grid, kThreads, 0, s>>>(b, group, pt)
            : k_assemble_tiles<8, false><<<grid, kThreads, 0, s>>>(b, group, pt);
    else if (b.d <= 16)
        tab ? k_assemble_tiles<16, true><<<grid, kThreads, 0, s>>>(b, group, pt)
            : k_assemble_tiles<16, false><<<grid, kThreads, 0, s>>>(b, group, pt);
    else
        k_assemble_tiles_generic<<<grid, kThreads, 0, s>>>(b, group);
    return cudaGetLastError();
}

cudaError_t launch_assemble_dense(int n, int d, const double* x, const double* theta, double p, int corr,
                                  double delta, double* R, cudaStream_t s) {
    dim3 grid((n + 255) / 256, n);
    k_assemble_dense<<<grid, 256, 0, s>>>(n, d, x, theta, p, corr, delta, R);
    return cudaGetLastError();
}

}  // namespace gp
