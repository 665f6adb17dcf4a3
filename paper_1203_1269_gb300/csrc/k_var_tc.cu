// k_var_tc.cu -- kriging means and variances from a resident fit with the
// variance's triangular solve on the tensor cores.
//
// For a test point x*: r_i = corr(x*, x_i) (eq. 2, no nugget), yhat =
// mu_hat + r'w, and with v = L^-1 r, a = L^-1 1
//   s2 = sigma2_hat [c0 - v'v + (1 - a'v)^2 / a'a]
// (Section 3 prices prediction at two triangular solves per point).  For N
// points and n design points v = L^-1 r is n^2 N multiply-adds, the one
// part of prediction that is GEMM-shaped.  Here it is a left-looking block
// forward substitution over the 128-row tile rows J of L, for 128 test
// points at a time (a point block, the rows of V):
//   C_J = R_J - sum_{K < J} V_K L_JK^T      (update: K = 128 J, split GEMM)
//   V_J = C_J W_J^T,  W_J = L_JJ^-1          (diagonal step: split GEMM)
// with v'v and a'v accumulated from each finished V_J.  Both products run
// as bf16 slice GEMMs (the Ozaki-style splitting of the factorisation's
// split path: an operand row scaled by 2^(7 - E) is cut into slices
// q_a 2^(-8a), |q_a| <= 128) with fp32 accumulation in tensor memory:
//   - the update with 5 slices of V and of L (15 products, groups a + b =
//     0, 1, 2 exact and >= 3 rounded, weight <= 2^-24).  V has one fixed
//     exponent: |v_i| <= ||v|| and v'v = r'R^-1 r <= c0 = 1 + delta, since
//     [R r; r' 1 + delta] is a correlation matrix plus delta I.  A group
//     sum stays exact in fp32 (below 2^24 in units of its weight) for K <
//     341 (3 pairs x 2^14 x K), so the accumulators are drained into
//     double-float registers every 320 columns of K;
//   - the diagonal step with 7 slices and every group exact (its error
//     scales with |C| |W|, which exceeds |V_J| when L_JJ is ill-conditioned),
//     in two 64-column halves (7 groups x 64 of the 512 tensor-memory
//     columns each).
// A CPU emulation of this arithmetic (the slicing, the dropped products,
// the fixed V exponent) against an FP64 substitution gave variance errors
// of 5e-11 .. 4e-10 sigma2 at n = 2048, d = 4 .. 10, cond(R) up to 5e8,
// against 2e-8 with 4 slices.
//
// r, its products with w (the mean) and the diagonal inverses come from
// kernels on the FP32 / FP64 pipes before the tensor-core pass:
//   k_var_w       W_J = L_JJ^-1 in double (one CTA per tile row), its rows'
//                 exponents and 7 slices
//   k_var_lmax,   row exponents and 5 slices of the rows of L left of the
//   k_var_lslice  diagonal (the update's B operand)
//   k_var_rhs     r for 128 points x 128 design points per CTA, in
//                 double-float as the assembly does, stored for the
//                 tensor-core pass, with the tile's partial r'w
//   k_var_mean    yhat from the partial sums, in tile-row order
//   k_var_tc      the persistent tensor-core pass: one CTA per SM walks
//                 point blocks; per block it runs J = 0 .. nt - 1
//
// All of it is rebuilt per call from the model (the tables take about 1 ms
// at n = 16384), so a model holds only its factor.
#include "corr.cuh"
#include "slices.cuh"

namespace gp {

namespace {

// 32 lanes x 32 bits x 4 columns of tensor memory
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kVarSlices = 5;                        // update operands
constexpr int kVarWSlices = GP_PANEL_SLICES;         // diagonal step operands (7)
constexpr uint32_t kHalfBytes = kChunkBytes / 2;     // 64 rows of a 128 x 32 chunk
// K chunks (of 32) between drains of the update's accumulators: the group of
// a + b = 2 (three slice pairs, |q_a q_b| <= 2^14) stays below 2^24 for 320
constexpr int kDrainChunks = 10;
static_assert(3 * 16384 * 32 * kDrainChunks < (1 << 24), "exact accumulator groups");
// The update's stages ahead of the ring whose operands the copy thread
// prefetches into L2: a stage's V slices come from HBM (each CTA streams its
// own block's V) and a two-slot ring of 80 KB stages alone leaves the
// tensor pipe waiting on that latency
constexpr int kPrefetch = 2;
static_assert(kPrefetch <= 4, "a prefetch reaches at most into the next tile row's first 4 chunks");

// Layouts (bf16 images of 128 x 32 chunks, as the factorisation's slices):
//   LS: row block J >= 1: [slice a][chunk k < 4J], first chunk 10 J (J - 1)
//   WS: block J: [slice a < 7][chunk k < 4]
//   VS (per CTA): [slice a][chunk k < 4 nt]
//   CS (per CTA): [slice a < 7][chunk k < 4]
__host__ __device__ inline size_t ls_chunk(int J, int a, int k) {
    return (size_t)10 * J * (J - 1) + (size_t)a * 4 * J + k;
}
__host__ __device__ inline size_t ls_chunks(int nt) { return (size_t)10 * nt * (nt - 1); }
__host__ __device__ inline size_t ws_chunk(int J, int a, int k) { return ((size_t)J * kVarWSlices + a) * 4 + k; }

// ------------------------------------------------------------ tables -------

// W_J = L_JJ^-1 by columns in double (thread j owns column j: W_jj =
// 1 / L_jj, W_ij = -(sum_{k=j}^{i-1} L_ik W_kj) / L_ii), then thread i
// cuts row i of W into 7 slices with its own exponent.  Dynamic shared
// memory: L_JJ packed (8256 doubles), W with row stride 129, 1 / L_ii.
constexpr int kWStride = GP_NB + 1;
constexpr size_t kVarWSmem = (size_t)(GP_NB * (GP_NB + 1) / 2 + GP_NB * kWStride + GP_NB) * sizeof(double);

__global__ void __launch_bounds__(GP_NB) k_var_w(const float2* L, int nt, __nv_bfloat16* WS, int* WE) {
    extern __shared__ double wsm[];
    double* Lp = wsm;                                  // L_rc at r (r + 1) / 2 + c
    double* W = Lp + GP_NB * (GP_NB + 1) / 2;          // W_ij at i * kWStride + j
    double* dinv = W + GP_NB * kWStride;
    const int J = blockIdx.x, j = threadIdx.x;
    const float2* T = L + (size_t)tile_index(J, J, nt) * GP_TILE_ELEMS;
    for (int c = 0; c < GP_NB; ++c)
        if (j >= c) Lp[j * (j + 1) / 2 + c] = (double)T[(size_t)c * GP_NB + j].x + (double)T[(size_t)c * GP_NB + j].y;
    __syncthreads();
    dinv[j] = 1.0 / Lp[j * (j + 1) / 2 + j];
    __syncthreads();
    for (int i = 0; i < GP_NB; ++i) {
        double w = 0.0;
        if (i == j) {
            w = dinv[j];
        } else if (i > j) {
            double s = 0.0;
            const double* Li = Lp + i * (i + 1) / 2;
            for (int k = j; k < i; ++k) s = fma(Li[k], W[k * kWStride + j], s);
            w = -s * dinv[i];
        }
        W[i * kWStride + j] = w;
    }
    __syncthreads();
    // row i = j of W: exponent from the high words, then the slices (the
    // same cut as the factorisation's panel slicing)
    const int i = j;
    float mx = 0.f;
    for (int k = 0; k <= i; ++k) mx = fmaxf(mx, fabsf(__double2float_rn(W[i * kWStride + k])));
    const int E = exponent_of(mx);
    WE[J * GP_NB + i] = E;
    float sa, sb;
    slice_scale(E, sa, sb);
    uint8_t* base = reinterpret_cast<uint8_t*>(WS + ws_chunk(J, 0, 0) * kChunkElems);
#pragma unroll 1
    for (int u = 0; u < 8; ++u) {
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const dfl x = df_from_double(W[i * kWStride + 16 * u + e]);
            v[e] = make_float2(x.hi, x.lo);
        }
        slice_pieces(v, sa, sb, i, 16 * (u & 1), kVarWSlices, base + (size_t)(u >> 1) * kChunkBytes,
                     (size_t)4 * kChunkBytes);
    }
}

// Largest |L_ik| (high words) of each row left of its diagonal block: tile
// (J, K), K < J, per CTA; the bits of non-negative floats order as ints.
__global__ void __launch_bounds__(GP_NB) k_var_lmax(const float2* L, int nt, int* lbits) {
    int J, K;
    tri_decode(blockIdx.x, J, K);   // J >= K over the strict lower triangle shifted by one
    J += 1;
    const int r = threadIdx.x;
    const float2* T = L + (size_t)tile_index(J, K, nt) * GP_TILE_ELEMS;
    float mx = 0.f;
    for (int c = 0; c < GP_NB; ++c) mx = fmaxf(mx, fabsf(T[(size_t)c * GP_NB + r].x));
    atomicMax(lbits + J * GP_NB + r, __float_as_int(mx));
}

// The 5 slices of tile (J, K), K < J, into row block J of LS; the CTA of
// K = 0 also stores the rows' exponents.  Thread (r, h) takes row r's
// columns 64 h .. 64 h + 63.
__global__ void __launch_bounds__(2 * GP_NB) k_var_lslice(const float2* L, int nt, const int* lbits,
                                                           __nv_bfloat16* LS, int* LE) {
    int J, K;
    tri_decode(blockIdx.x, J, K);
    J += 1;
    const int r = threadIdx.x & (GP_NB - 1), h = threadIdx.x >> 7;
    const float2* T = L + (size_t)tile_index(J, K, nt) * GP_TILE_ELEMS;
    const int E = exponent_of(__int_as_float(lbits[J * GP_NB + r]));
    if (K == 0 && h == 0) LE[J * GP_NB + r] = E;
    float sa, sb;
    slice_scale(E, sa, sb);
    uint8_t* base = reinterpret_cast<uint8_t*>(LS + ls_chunk(J, 0, 4 * K) * kChunkElems);
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
        const int c0 = 64 * h + 16 * u;
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = T[(size_t)(c0 + e) * GP_NB + r];
        slice_pieces(v, sa, sb, r, c0 & 31, kVarSlices, base + (size_t)(c0 >> 5) * kChunkBytes,
                     (size_t)4 * J * kChunkBytes);
    }
}

// --------------------------------------------------------------- r ---------

// |dx|^p for a general p without a logarithm or an exponential (the
// table-driven reduction of P. T. P. Tang, ACM TOMS 16 (1990), applied to
// the power): |dx| = 2^m F_j (1 + u), F_j = 1 + j/kPowN the table point
// nearest to the mantissa (|u| <= 2^-8), so that
//   theta_k |dx|^p = [theta_k 2^(m p)] F_j^p (1 + u)^p
// with 2^(m p) (m = -kPowM .. kPowM) and F_j^p from tables in double-float
// and (1 + u)^p by its binomial series to u^5 (the u^6 term is below
// 2^-53 for p in (0, 2]).  The tables depend on p alone and are built once
// per call (k_var_rhs_tables), with the exponential's 2^(-j/1024).
constexpr int kPowNBits = 7;
constexpr int kPowN = 1 << kPowNBits;
constexpr int kPowM = 60;                            // |dx| in [2^-60, 2^60]
constexpr int kPowMs = 2 * kPowM + 1;
constexpr int kPowMaxD = 16;                         // above: the general routine per term
// the table image, in float2 units: 2^(-j/1024), 2^(m p), F_j^p, then
// 1/F_j as floats
constexpr int kTabExp = 0;
constexpr int kTabTwo = kExpTab;
constexpr int kTabF = kTabTwo + kPowMs;
constexpr int kTabInv = kTabF + kPowN;
constexpr int kTabLen = kTabInv + kPowN / 2;

__global__ void k_var_rhs_tables(double p, float2* tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v;
    if (i < kTabTwo) {
        v = exp2(-(double)i / (double)kExpTab);      // as fill_exp2_table
    } else if (i < kTabF) {
        v = exp2((double)(i - kTabTwo - kPowM) * p);
    } else if (i < kTabInv) {
        v = pow(1.0 + (double)(i - kTabF) / kPowN, p);
    } else {
        if (i < kTabInv + kPowN)
            reinterpret_cast<float*>(tab + kTabInv)[i - kTabInv] =
                (float)(1.0 / (1.0 + (double)(i - kTabInv) / kPowN));
        return;
    }
    const dfl t = df_from_double(v);
    tab[i] = make_float2(t.hi, t.lo);
}

// (1 + u)^p = 1 + p u + c2 u^2 + (c3 + c4 u + c5 u^2) u^3 for u = uh + ul,
// |u| <= 2^-8, |ul| <= 2^-24 (it carries the argument's low word): p u and
// c2 u^2 as exact products of the high words plus their cross terms, the
// rest in float (it is below 2^-26) with u^3 = uh^2 (uh + 3 ul)
__device__ __forceinline__ dfl pow_series(float uh, float ul, dfl pd, dfl c2, float c3, float c4, float c5) {
    const float t1 = __fmul_rn(pd.hi, uh);
    float t1e = __fmaf_rn(pd.hi, uh, -t1);
    t1e = __fmaf_rn(pd.hi, ul, t1e);
    t1e = __fmaf_rn(pd.lo, uh, t1e);
    const float sq = __fmul_rn(uh, uh);
    float sqe = __fmaf_rn(uh, uh, -sq);
    sqe = __fmaf_rn(__fadd_rn(uh, uh), ul, sqe);
    const float t2 = __fmul_rn(c2.hi, sq);
    float t2e = __fmaf_rn(c2.hi, sq, -t2);
    t2e = __fmaf_rn(c2.hi, sqe, t2e);
    t2e = __fmaf_rn(c2.lo, sq, t2e);
    float q = __fmaf_rn(uh, c5, c4);
    q = __fmaf_rn(uh, q, c3);
    const float t3 = __fmul_rn(__fmul_rn(sq, __fmaf_rn(3.f, ul, uh)), q);
    float a, al, b, bl;
    fast_two_sum(1.f, t1, a, al);
    fast_two_sum(a, t2, b, bl);
    const float lo = __fadd_rn(__fadd_rn(al, bl), __fadd_rn(__fadd_rn(t1e, t2e), t3));
    dfl P;
    fast_two_sum(b, lo, P.hi, P.lo);
    return P;
}

// theta_k |x|^p for x = (xh, xl), 2^-60 <= xh <= 2^60, from the tables:
// thm = theta_k 2^(m p) for this k (indexed by m + kPowM), fp = F_j^p,
// inv = 1/F_j (rounded; the residual of the division is formed exactly)
__device__ __forceinline__ dfl pow_tab(float xh, float xl, const dfl* thm, const dfl* fp, const float* inv,
                                       dfl pd, dfl c2, float c3, float c4, float c5, dfl& P) {
    const int rb = __float_as_int(xh) + (1 << (22 - kPowNBits));   // mantissa rounded to kPowNBits bits
    const int e = rb >> 23;                                          // biased exponent of 2^m F_j
    const int j = (rb >> (23 - kPowNBits)) & (kPowN - 1);
    const float Fm = __int_as_float(rb & ~((1 << (23 - kPowNBits)) - 1));   // 2^m F_j
    const float g = __int_as_float((254 - e) << 23);                          // 2^-m
    const float fh = __fmul_rn(__fsub_rn(xh, Fm), g);                        // exact (Sterbenz)
    const float fl = __fmul_rn(xl, g);
    const float F = __fmul_rn(Fm, g);
    const float iv = inv[j];
    const float uh = __fmul_rn(fh, iv);
    const float ul = __fmul_rn(__fadd_rn(__fmaf_rn(-uh, F, fh), fl), iv);
    P = pow_series(uh, ul, pd, c2, c3, c4, c5);
    return df_mul(thm[e - 127 + kPowM], fp[j]);
}

struct RhsArgs {
    int n, d, nt, N, m0;          // m0: first point of the launch (point block 0)
    const float2* x;              // n x d design points (double-float)
    const double* theta;
    double p;
    int corr;
    const double* xs;             // N x d test points
    const float2* w;              // npad: R^-1 (Y - 1 mu_hat)
    float2* RX;                   // [pb][npad][128] or null (mean only)
    float2* MP;                   // [pb][nt][128] partial r'w
    const float2* tab;            // k_var_rhs_tables' image
    int tabpow;                   // 1: general p, power-exponential, d <= kPowMaxD
    double c2;                    // binomial coefficients of (1 + u)^p
    float c3, c4, c5;
};

// r for point block blockIdx.y (128 points) and tile row blockIdx.x (128
// design points) in double-float: S = sum_k theta_k |dx_k|^p (compensated,
// in dimension order), r = exp(-S) (times the Matern polynomials).  A
// general p on the power-exponential family takes the powers from the
// tables (pow_tab) and sums S as the assembly does (one TwoSum per term
// on the high words, all terms being >= 0); p = 1, 2, the Matern family and
// d > kPowMaxD form each term as the assembly's double-float routines do.
// Thread (r, h) takes design points h, h + 2, ..., so one warp writes 32
// consecutive points of one design point.  Dynamic shared memory: the
// points' coordinates [d][128], the design points' [128][d], theta, the
// exp table, and with the tables theta_k 2^(m p) [d][kPowMs], F_j^p and 1/F_j.
// DB > 0: d = DB exactly (the table path's d <= kPowMaxD), so that the loop
// over the dimensions has a constant bound; DB = 0: d at run time.
template <int DB>
__global__ void __launch_bounds__(2 * GP_NB) k_var_rhs(RhsArgs g) {
    extern __shared__ dfl rsm[];
    const int d = DB > 0 ? DB : g.d;
    dfl* xsT = rsm;                        // [d][128]
    dfl* xd = xsT + d * GP_NB;             // [128][d]
    dfl* th = xd + GP_NB * d;              // [d]
    dfl* tab = th + d;                     // [kExpTab]
    dfl* thm = tab + kExpTab;              // [d][kPowMs]   (tabpow)
    dfl* fp = thm + d * kPowMs;            // [kPowN]        (tabpow)
    float* inv = reinterpret_cast<float*>(fp + kPowN);   // [kPowN] (tabpow)
    __shared__ dfl part[2][GP_NB];
    const int J = blockIdx.x, pb = blockIdx.y;
    const int mb = g.m0 + pb * GP_NB;
    const bool tabpow = g.tabpow != 0;
    for (int q = threadIdx.x; q < GP_NB * d; q += blockDim.x) {
        const int m = q / d, k = q % d;
        xsT[k * GP_NB + m] = (mb + m < g.N) ? df_from_double(g.xs[(size_t)(mb + m) * d + k]) : dfl{0.f, 0.f};
        const int i = J * GP_NB + m;
        xd[q] = (i < g.n) ? df_load(g.x + (size_t)i * d + k) : dfl{0.f, 0.f};
    }
    for (int q = threadIdx.x; q < d; q += blockDim.x) th[q] = df_from_double(corr_theta_scale(g.corr) * g.theta[q]);
    for (int q = threadIdx.x; q < kExpTab; q += blockDim.x) tab[q] = df_load(g.tab + kTabExp + q);
    if (tabpow) {
        for (int q = threadIdx.x; q < kPowN; q += blockDim.x) {
            fp[q] = df_load(g.tab + kTabF + q);
            inv[q] = reinterpret_cast<const float*>(g.tab + kTabInv)[q];
        }
        __syncthreads();                   // th
        for (int q = threadIdx.x; q < d * kPowMs; q += blockDim.x)
            thm[q] = df_mul(th[q / kPowMs], df_load(g.tab + kTabTwo + q % kPowMs));
    }
    __syncthreads();
    const dfl pd = df_from_double(g.p);
    const bool matern = corr_is_matern(g.corr);
    const int pmode = matern ? kPowOne : pow_mode(g.p);
    const dfl third = df_from_double(1.0 / 3.0);
    const dfl c2 = df_from_double(g.c2);
    const int r = threadIdx.x & (GP_NB - 1), h = threadIdx.x >> 7;
    const bool point_ok = mb + r < g.N;
    float2* out = g.RX ? g.RX + ((size_t)pb * g.nt * GP_NB + (size_t)J * GP_NB) * GP_NB + r : nullptr;
    dfl mean = {0.f, 0.f};
    if (tabpow) {
        for (int c = h; c < GP_NB; c += 2) {
            const int i = J * GP_NB + c;
            dfl v = {0.f, 0.f};
            if (point_ok && i < g.n) {
                float sh = 0.f, sl = 0.f;
#pragma unroll
                for (int k = 0; k < d; ++k) {
                    dfl dx = df_sub(xsT[k * GP_NB + r], xd[c * d + k]);
                    if (dx.hi < 0.f) dx = df_neg(dx);
                    dfl A, P;
                    if (dx.hi >= 0x1p-60f && dx.hi <= 0x1p60f) {
                        A = pow_tab(dx.hi, dx.lo, thm + k * kPowMs, fp, inv, pd, c2, g.c3, g.c4, g.c5, P);
                    } else {
                        A = df_mul(th[k], df_powabs(dx, kPowGeneral, g.p, pd, tab));   // 0 at dx = 0
                        P = {1.f, 0.f};
                    }
                    // theta_k |dx_k|^p = A P into S
                    const float ph = __fmul_rn(A.hi, P.hi);
                    sl = __fadd_rn(sl, __fmaf_rn(A.hi, P.hi, -ph));
                    sl = __fmaf_rn(A.hi, P.lo, sl);
                    sl = __fmaf_rn(A.lo, P.hi, sl);
                    float s2, e2;
                    two_sum(sh, ph, s2, e2);
                    sh = s2;
                    sl = __fadd_rn(sl, e2);
                }
                dfl S;
                fast_two_sum(sh, sl, S.hi, S.lo);
                v = df_exp_neg(S, tab);
                mean = df_fma(v, df_load(g.w + i), mean);
            }
            if (out) out[(size_t)c * GP_NB] = make_float2(v.hi, v.lo);
        }
    } else {
        for (int c = h; c < GP_NB; c += 2) {
            const int i = J * GP_NB + c;
            dfl v = {0.f, 0.f};
            if (point_ok && i < g.n) {
                dfl s = {0.f, 0.f}, qp = {1.f, 0.f};
                for (int k = 0; k < d; ++k) {
                    const dfl dx = df_sub(xsT[k * GP_NB + r], xd[c * d + k]);
                    const dfl hk = df_mul(th[k], df_powabs(dx, pmode, g.p, pd, tab));
                    s = df_add(s, hk);
                    if (matern) qp = df_mul(qp, matern_q_df(hk, g.corr, third));
                }
                v = df_exp_neg(s, tab);
                if (matern) v = df_mul(v, qp);
                mean = df_fma(v, df_load(g.w + i), mean);
            }
            if (out) out[(size_t)c * GP_NB] = make_float2(v.hi, v.lo);
        }
    }
    part[h][r] = mean;
    __syncthreads();
    if (h == 0) {
        const dfl m = df_add(part[0][r], part[1][r]);
        g.MP[((size_t)pb * g.nt + J) * GP_NB + r] = make_float2(m.hi, m.lo);
    }
}

// yhat = mu_hat + sum_J MP[J] in tile-row order (the same bits with or
// without variances)
__global__ void k_var_mean(const float2* MP, int nt, int N, int m0, int npb, const double* sc, double* yhat) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npb * GP_NB) return;
    const int pb = t / GP_NB, r = t % GP_NB;
    if (m0 + t >= N) return;
    dfl s = {0.f, 0.f};
    for (int J = 0; J < nt; ++J) s = df_add(s, df_load(MP + ((size_t)pb * nt + J) * GP_NB + r));
    yhat[m0 + t] = sc[1] + df_to_double(s);
}

// ------------------------------------------------------ tensor cores -------

struct VarArgs {
    int nt, npb, N, m0;           // tile rows; point blocks, points in all, first point of this launch
    int ev;                       // the fixed exponent of V's rows
    const __nv_bfloat16* LS;
    const int* LE;                // npad
    const __nv_bfloat16* WS;
    const int* WE;                // npad
    const float2* a;              // npad: L^-1 1
    const double* sc;             // model scalars: sigma2_hat at 2, a'a at 5
    double c0;
    const float2* RX;             // [pb][npad][128]
    __nv_bfloat16* VS;            // per CTA, vs_stride elements
    __nv_bfloat16* CS;            // per CTA, cs_stride elements
    size_t vs_stride, cs_stride;
    double* s2;
    int* err;
    int inject_timeout;           // test hook: CTA 0 waits 5 ms on a barrier nothing signals
};

// Warp 0 copies, warp 1 issues the MMAs and owns the tensor memory, warps
// 2 and 3 idle, warps 4 .. 19 are the epilogue (a tensor-memory lane
// quarter and a quarter of the columns each).  Registers: 48 for
// warpgroup 0 (the fully unrolled MMA issue of the 7-slice step spills at
// 32), 104 for the epilogue, out of 640 threads x 96 at launch.
constexpr int kVarThreads = 640;
constexpr int kVarEpiThreads = 512;
constexpr int kVarRegsLow = 48;
constexpr int kVarRegsHigh = 104;
static_assert(128 * kVarRegsLow + kVarEpiThreads * kVarRegsHigh <= kVarThreads * 96, "register split");
// one ring slot holds the larger of the two stages: 5 + 5 chunks (update)
// or 7 chunks and 7 half chunks (diagonal step)
constexpr uint32_t kVarStageBytes = kVarWSlices * (kChunkBytes + kHalfBytes);
static_assert(kVarStageBytes >= 2 * kVarSlices * kChunkBytes, "stage slot");
constexpr size_t kVarSmem = 2 * (size_t)kVarStageBytes + 1024;

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The MMAs of one stage: every slice product (a, b), a + b < NS, over the
// stage's two K = 16 steps, into group min(a + b, NG - 1); in the first
// stage after a drain the first product of each group overwrites it.
template <int NS, int NG, int NT, uint32_t kBBytes, bool FIRST>
__device__ __forceinline__ void var_issue(uint32_t tacc, uint64_t ad0, uint64_t bd0, uint32_t idesc) {
#pragma unroll
    for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int bb = 0; a + bb < NS; ++bb) {
            const int gr = (a + bb < NG - 1) ? (a + bb) : (NG - 1);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint64_t ad = ad0 + (uint64_t)((a * kChunkBytes + kk * 32) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((bb * kBBytes + kk * 32) >> 4);
                const bool overwrite = FIRST && a == 0 && kk == 0 && bb <= NG - 1;
                mma_bf16(tacc + gr * NT, ad, bd, idesc, overwrite ? 0u : 1u);
            }
        }
    }
}

__global__ void __launch_bounds__(kVarThreads, 1) k_var_tc(VarArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(8) uint64_t tfull_bar, tempty_bar;
    __shared__ __align__(8) uint64_t cs_bar, v_bar, row_bar, red_bar;
    __shared__ __align__(8) uint64_t drain_bar, never_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int blocks_done;
    __shared__ float pmax[2][4][GP_NB];
    __shared__ dfl red[2][2][4][GP_NB];

    const int nt = g.nt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tfull_bar, 1);
        mbar_init(&tempty_bar, kVarEpiThreads);
        mbar_init(&cs_bar, kVarEpiThreads);
        mbar_init(&v_bar, kVarEpiThreads);
        mbar_init(&row_bar, kVarEpiThreads);
        mbar_init(&red_bar, kVarEpiThreads);
        mbar_init(&drain_bar, 1);
        mbar_init(&never_bar, 1);
        abort_flag = 0;
        blocks_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;
    const uint8_t* VSb = reinterpret_cast<const uint8_t*>(g.VS + (size_t)blockIdx.x * g.vs_stride);
    const uint8_t* CSb = reinterpret_cast<const uint8_t*>(g.CS + (size_t)blockIdx.x * g.cs_stride);

    if (warp >= 4) {
        regs_inc<kVarRegsHigh>();
        // ------------------------------------------------------ epilogue --
        const int q = warp & 3, part = (warp - 4) >> 2, row = 32 * q + lane;
        const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
        uint8_t* vs = const_cast<uint8_t*>(VSb);
        uint8_t* cs = const_cast<uint8_t*>(CSb);
        float sav, sbv;
        slice_scale(g.ev, sav, sbv);
        int use = 0, steps = 0, blocks = 0;
        bool ok = true;
        for (int pb = blockIdx.x; ok && pb < g.npb; pb += gridDim.x) {
            dfl vv = {0.f, 0.f}, av = {0.f, 0.f};
            const float2* rx = g.RX + (size_t)pb * nt * GP_NB * GP_NB + row;
            for (int J = 0; ok && J < nt; ++J) {
                // update: S = sum over the drained K blocks of V_K L_JK^T, kept
                // unscaled (the scale 2^(ev + E_L - 14) of a column is a power
                // of two, the same in every drain: applied once at the end)
                float2 c[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) c[j] = make_float2(0.f, 0.f);
                for (int k0 = 0; k0 < 4 * J; k0 += kDrainChunks) {
                    if (!mbar_wait(&tfull_bar, use & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int cb = 0; cb < 8; ++cb) {
                        float d[4][4];
#pragma unroll
                        for (int gg = 0; gg < 4; ++gg) tmem_ld4(lane_addr + gg * GP_NB + 32 * part + 4 * cb, d[gg]);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            // groups 0 .. 2 exact, group 3 (weight <= 2^-24)
                            // rounded, straight into the running double-float
                            // sum, renormalised once per drain
                            float h, l, e2, s, t;
                            two_sum(d[0][j], d[1][j], h, l);
                            two_sum(h, d[2][j], h, e2);
                            l = __fadd_rn(__fadd_rn(l, e2), d[3][j]);
                            two_sum(c[4 * cb + j].x, h, s, t);
                            t = __fadd_rn(c[4 * cb + j].y, __fadd_rn(t, l));
                            two_sum(s, t, s, t);
                            c[4 * cb + j] = make_float2(s, t);
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&tempty_bar);
                    ++use;
                }
                if (!ok) break;
                // C_J = R_J - S; the row's exponent over its four column parts
                float mx = 0.f;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float2 rv = rx[(size_t)(J * GP_NB + 32 * part + j) * GP_NB];
                    float sc = 0.f;
                    if (J > 0) {
                        const int e = g.ev + __ldg(g.LE + J * GP_NB + 32 * part + j) - 14;
                        sc = (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
                    }
                    const dfl t = df_sub(dfl{rv.x, rv.y}, dfl{__fmul_rn(c[j].x, sc), __fmul_rn(c[j].y, sc)});
                    c[j] = make_float2(t.hi, t.lo);
                    mx = fmaxf(mx, fabsf(t.hi));
                }
                pmax[steps & 1][part][row] = mx;
                mbar_arrive(&row_bar);
                if (!mbar_wait(&row_bar, steps & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                mx = fmaxf(fmaxf(pmax[steps & 1][0][row], pmax[steps & 1][1][row]),
                           fmaxf(pmax[steps & 1][2][row], pmax[steps & 1][3][row]));
                ++steps;
                const int E = exponent_of(mx);
                {
                    float sa, sb;
                    slice_scale(E, sa, sb);
                    float2 lo16[16], hi16[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        lo16[j] = c[j];
                        hi16[j] = c[16 + j];
                    }
                    slice_pieces(lo16, sa, sb, row, 0, kVarWSlices, cs + (size_t)part * kChunkBytes,
                                 (size_t)4 * kChunkBytes);
                    slice_pieces(hi16, sa, sb, row, 16, kVarWSlices, cs + (size_t)part * kChunkBytes,
                                 (size_t)4 * kChunkBytes);
                }
                fence_proxy_async_global();
                mbar_arrive(&cs_bar);
                // diagonal step, two 64-column halves: V_J = C_J W_J^T
                for (int hf = 0; hf < 2; ++hf) {
                    if (!mbar_wait(&tfull_bar, use & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    float2 vb[16];
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb) {
                        float d[kVarWSlices][4];
#pragma unroll
                        for (int gg = 0; gg < kVarWSlices; ++gg)
                            tmem_ld4(lane_addr + gg * 64 + 16 * part + 4 * cb, d[gg]);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            // every group exact in the double-float sum
                            float h, l;
                            two_sum(d[0][j], d[1][j], h, l);
#pragma unroll
                            for (int gg = 2; gg < kVarWSlices; ++gg) {
                                float s2, e2;
                                two_sum(h, d[gg][j], s2, e2);
                                l = __fadd_rn(l, e2);
                                fast_two_sum(s2, l, h, l);
                            }
                            const int col = J * GP_NB + 64 * hf + 16 * part + 4 * cb + j;
                            const int e = E + __ldg(g.WE + col) - 14;
                            const float sc = (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
                            dfl v;
                            fast_two_sum(__fmul_rn(h, sc), __fmul_rn(l, sc), v.hi, v.lo);
                            vv = df_fma(v, v, vv);
                            av = df_fma(df_load(g.a + col), v, av);
                            vb[4 * cb + j] = make_float2(v.hi, v.lo);
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&tempty_bar);
                    ++use;
                    // V_J's slices for the later tile rows: chunk 4 J + 2 hf + part / 2
                    slice_pieces(vb, sav, sbv, row, 16 * (part & 1), kVarSlices,
                                 vs + (size_t)(4 * J + 2 * hf + (part >> 1)) * kChunkBytes,
                                 (size_t)4 * nt * kChunkBytes);
                }
                if (!ok) break;
                fence_proxy_async_global();
                mbar_arrive(&v_bar);
            }
            if (!ok) break;
            // v'v and a'v of the point over the four column parts
            red[blocks & 1][0][part][row] = vv;
            red[blocks & 1][1][part][row] = av;
            mbar_arrive(&red_bar);
            if (!mbar_wait(&red_bar, blocks & 1, &abort_flag)) {
                ok = false;
                break;
            }
            if (part == 0) {
                const int m = g.m0 + pb * GP_NB + row;
                if (m < g.N) {
                    dfl s[2];
#pragma unroll
                    for (int k = 0; k < 2; ++k)
                        s[k] = df_add(df_add(red[blocks & 1][k][0][row], red[blocks & 1][k][1][row]),
                                      df_add(red[blocks & 1][k][2][row], red[blocks & 1][k][3][row]));
                    const double gg = 1.0 - df_to_double(s[1]);
                    g.s2[m] = g.sc[2] * (g.c0 - df_to_double(s[0]) + gg * gg / g.sc[5]);
                }
            }
            ++blocks;
            if (threadIdx.x == 4 * 32) blocks_done = blocks;
        }
        if (!ok) abort_flag = 1;
    } else {
        regs_dec<kVarRegsLow>();
        if (warp == 0 && lane == 0) {
            // ------------------------------------------------- copies --
            int gs = 0, csn = 0, vn = 0;
            bool ok = true;
            auto stage = [&](int nA, const uint8_t* srcA, size_t strideA, int nB, const uint8_t* srcB,
                             size_t strideB, uint32_t bBytes) -> bool {
                const int st = gs & 1;
                if (gs >= 2 && !mbar_wait(&empty_bar[st], ((gs >> 1) - 1) & 1, &abort_flag)) return false;
                uint8_t* sa = smem + st * kVarStageBytes;
                uint8_t* sb = sa + (size_t)nA * kChunkBytes;
                mbar_expect_tx(&full_bar[st], (uint32_t)nA * kChunkBytes + (uint32_t)nB * bBytes);
                for (int a = 0; a < nA; ++a) bulk_g2s(sa + (size_t)a * kChunkBytes, srcA + a * strideA, kChunkBytes, &full_bar[st]);
                for (int a = 0; a < nB; ++a) bulk_g2s(sb + (size_t)a * bBytes, srcB + a * strideB, bBytes, &full_bar[st]);
                ++gs;
                return true;
            };
            const uint8_t* LSb = reinterpret_cast<const uint8_t*>(g.LS);
            const uint8_t* WSb = reinterpret_cast<const uint8_t*>(g.WS);
            for (int pb = blockIdx.x; ok && pb < g.npb; pb += gridDim.x) {
                for (int J = 0; ok && J < nt; ++J) {
                    for (int k = 0; ok && k < 4 * J; ++k) {
                        if (k == 4 * (J - 1)) {
                            // V_{J-1}'s slices, written by the epilogue in the previous tile row
                            if (!mbar_wait(&v_bar, vn & 1, &abort_flag)) {
                                ok = false;
                                break;
                            }
                            ++vn;
                        }
                        {
                            // L2 prefetch of chunk k + kPrefetch, or of the next
                            // tile row's first chunks (a hint: L2 stays coherent
                            // with the epilogue's later writes of V)
                            int kp = k + kPrefetch, Jp = J;
                            if (kp >= 4 * J) {
                                kp -= 4 * J;
                                Jp = J + 1;
                            }
                            if (Jp < nt)
                                for (int a = 0; a < kVarSlices; ++a) {
                                    prefetch_l2(VSb + ((size_t)a * 4 * nt + kp) * kChunkBytes, kChunkBytes);
                                    prefetch_l2(LSb + ls_chunk(Jp, a, kp) * kChunkBytes, kChunkBytes);
                                }
                        }
                        ok = stage(kVarSlices, VSb + (size_t)k * kChunkBytes, (size_t)4 * nt * kChunkBytes,
                                   kVarSlices, LSb + ls_chunk(J, 0, k) * kChunkBytes, (size_t)4 * J * kChunkBytes,
                                   kChunkBytes);
                    }
                    if (!ok) break;
                    if (!mbar_wait(&cs_bar, csn & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    ++csn;
                    for (int hf = 0; ok && hf < 2; ++hf)
                        for (int k = 0; ok && k < 4; ++k)
                            ok = stage(kVarWSlices, CSb + (size_t)k * kChunkBytes, (size_t)4 * kChunkBytes,
                                       kVarWSlices, WSb + ws_chunk(J, 0, k) * kChunkBytes + hf * kHalfBytes,
                                       (size_t)4 * kChunkBytes, kHalfBytes);
                }
                // the last tile row's V slices: every phase of v_bar is taken in order
                if (ok && !mbar_wait(&v_bar, vn & 1, &abort_flag)) ok = false;
                ++vn;
            }
            if (!ok) abort_flag = 1;
            // no copy may still be landing when the CTA retires
            for (int k = (gs > 2 ? gs - 2 : 0); k < gs; ++k) mbar_wait(&full_bar[k & 1], (k >> 1) & 1);
        } else if (warp == 1 && lane == 0) {
            // --------------------------------------------------- MMAs --
            int gs = 0, use = 0;
            bool ok = true;
            constexpr uint32_t idesc_u = idesc_bf16(GP_NB), idesc_w = idesc_bf16(64);
            if (g.inject_timeout && blockIdx.x == 0 && !mbar_wait(&never_bar, 0, &abort_flag, 5000000ull)) ok = false;
            auto tmem_free = [&]() -> bool {
                if (use >= 1 && !mbar_wait(&tempty_bar, (use - 1) & 1, &abort_flag)) return false;
                tc_fence_after();
                return true;
            };
            auto take = [&](uint32_t& sa) -> bool {
                const int st = gs & 1;
                if (!mbar_wait(&full_bar[st], (gs >> 1) & 1, &abort_flag)) return false;
                tc_fence_after();
                sa = smem_u32(smem + st * kVarStageBytes);
                return true;
            };
            for (int pb = blockIdx.x; ok && pb < g.npb; pb += gridDim.x) {
                for (int J = 0; ok && J < nt; ++J) {
                    for (int k0 = 0; ok && k0 < 4 * J; k0 += kDrainChunks) {
                        if (!(ok = tmem_free())) break;
                        const int k1 = (k0 + kDrainChunks < 4 * J) ? k0 + kDrainChunks : 4 * J;
                        for (int k = k0; k < k1; ++k) {
                            uint32_t sa;
                            if (!(ok = take(sa))) break;
                            const uint64_t ad0 = smem_desc(sa, 16, 512, 4);
                            const uint64_t bd0 = smem_desc(sa + kVarSlices * kChunkBytes, 16, 512, 4);
                            if (k == k0) var_issue<kVarSlices, 4, GP_NB, kChunkBytes, true>(tbase, ad0, bd0, idesc_u);
                            else         var_issue<kVarSlices, 4, GP_NB, kChunkBytes, false>(tbase, ad0, bd0, idesc_u);
                            mma_commit(&empty_bar[gs & 1]);
                            ++gs;
                        }
                        if (!ok) break;
                        mma_commit(&tfull_bar);
                        ++use;
                    }
                    for (int hf = 0; ok && hf < 2; ++hf) {
                        if (!(ok = tmem_free())) break;
                        for (int k = 0; k < 4; ++k) {
                            uint32_t sa;
                            if (!(ok = take(sa))) break;
                            const uint64_t ad0 = smem_desc(sa, 16, 512, 4);
                            const uint64_t bd0 = smem_desc(sa + kVarWSlices * kChunkBytes, 16, 512, 4);
                            if (k == 0) var_issue<kVarWSlices, kVarWSlices, 64, kHalfBytes, true>(tbase, ad0, bd0, idesc_w);
                            else        var_issue<kVarWSlices, kVarWSlices, 64, kHalfBytes, false>(tbase, ad0, bd0, idesc_w);
                            mma_commit(&empty_bar[gs & 1]);
                            ++gs;
                        }
                        if (!ok) break;
                        mma_commit(&tfull_bar);
                        ++use;
                    }
                }
            }
            if (!ok) abort_flag = 1;
            // every MMA issued has completed before tensor memory is released
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_flag) {
        // the point blocks this CTA had not finished read NaN
        if (threadIdx.x == 0) atomicExch(g.err, GP_ETIMEOUT);
        if (threadIdx.x < GP_NB)
            for (int pb = blockIdx.x + blocks_done * gridDim.x; pb < g.npb; pb += gridDim.x) {
                const int m = g.m0 + pb * GP_NB + threadIdx.x;
                if (m < g.N) g.s2[m] = __longlong_as_double(0x7ff8000000000000ll);
            }
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

}  // namespace

// ------------------------------------------------------------- host --------

size_t var_table_bytes(int nt) {
    const size_t npad = (size_t)nt * GP_NB;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return al(ls_chunks(nt) * kChunkBytes) + al((size_t)nt * kVarWSlices * 4 * kChunkBytes) + 3 * al(npad * sizeof(int));
}
size_t var_rx_bytes(int nt) { return (size_t)nt * GP_NB * GP_NB * sizeof(float2); }
size_t var_mp_bytes(int nt) { return (size_t)nt * GP_NB * sizeof(float2); }
size_t var_vs_bytes(int nt) { return (size_t)kVarSlices * 4 * nt * kChunkBytes; }
size_t var_cta_bytes(int nt) { return var_vs_bytes(nt) + (size_t)kVarWSlices * 4 * kChunkBytes; }

VarTables var_tables_at(void* base, int nt) {
    const size_t npad = (size_t)nt * GP_NB;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char* c = static_cast<char*>(base);
    VarTables t;
    t.LS = reinterpret_cast<__nv_bfloat16*>(c); c += al(ls_chunks(nt) * kChunkBytes);
    t.WS = reinterpret_cast<__nv_bfloat16*>(c); c += al((size_t)nt * kVarWSlices * 4 * kChunkBytes);
    t.LE = reinterpret_cast<int*>(c); c += al(npad * sizeof(int));
    t.WE = reinterpret_cast<int*>(c); c += al(npad * sizeof(int));
    t.lbits = reinterpret_cast<int*>(c);
    return t;
}

// The slices of W_J (all J) and of the rows of L left of their diagonal
// blocks: 1 + (nt > 1 ? 2 : 0) kernels.
cudaError_t launch_var_tables(const float2* L, int nt, const VarTables& t, cudaStream_t s, int* kernels) {
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_var_w, kVarWSmem, attr);
    if (e != cudaSuccess) return e;
    k_var_w<<<nt, GP_NB, kVarWSmem, s>>>(L, nt, t.WS, t.WE);
    *kernels = 1;
    if ((e = cudaGetLastError()) != cudaSuccess || nt == 1) return e;
    const unsigned tiles = (unsigned)((long long)nt * (nt - 1) / 2);
    if ((e = cudaMemsetAsync(t.lbits, 0, (size_t)nt * GP_NB * sizeof(int), s)) != cudaSuccess) return e;
    k_var_lmax<<<tiles, GP_NB, 0, s>>>(L, nt, t.lbits);
    k_var_lslice<<<tiles, 2 * GP_NB, 0, s>>>(L, nt, t.lbits, t.LS, t.LE);
    *kernels = 3;
    return cudaGetLastError();
}

// The tensor-core kernel raises its epilogue warps to kVarRegsHigh
// registers, which completes only if the block was launched with enough
// registers for the whole split: checked once per device.
static bool var_tc_fits() {
    static std::atomic<int> ok[kMaxDevices];   // 0 unknown, 1 yes, 2 no
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < kMaxDevices;
    int v = cached ? ok[dev].load(std::memory_order_relaxed) : 0;
    if (v == 0) {
        cudaFuncAttributes fa{};
        v = 2;
        if (cudaFuncGetAttributes(&fa, k_var_tc) == cudaSuccess &&
            128 * kVarRegsLow + kVarEpiThreads * kVarRegsHigh <= kVarThreads * fa.numRegs &&
            fa.maxThreadsPerBlock >= kVarThreads)
            v = 1;
        cudaGetLastError();
        if (cached) ok[dev].store(v, std::memory_order_relaxed);
    }
    return v == 1;
}

// r and the partial means of npb point blocks from point m0 (RX null: means
// only), then yhat: 2 kernels.
// k_var_rhs for one d (0: any), its shared-memory limit raised once per
// device and size
template <int DB>
static cudaError_t launch_rhs(dim3 grid, size_t smem, cudaStream_t s, const RhsArgs& r) {
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_var_rhs<DB>, smem, attr);
    if (e != cudaSuccess) return e;
    k_var_rhs<DB><<<grid, 2 * GP_NB, smem, s>>>(r);
    return cudaGetLastError();
}

static cudaError_t launch_rhs_exact(int d, dim3 grid, size_t smem, cudaStream_t s, const RhsArgs& r) {
    switch (d) {
#define GP_RHS_EXACT(D) \
        case D: return launch_rhs<D>(grid, smem, s, r)
        GP_RHS_EXACT(1); GP_RHS_EXACT(2); GP_RHS_EXACT(3); GP_RHS_EXACT(4);
        GP_RHS_EXACT(5); GP_RHS_EXACT(6); GP_RHS_EXACT(7); GP_RHS_EXACT(8);
        GP_RHS_EXACT(9); GP_RHS_EXACT(10); GP_RHS_EXACT(11); GP_RHS_EXACT(12);
        GP_RHS_EXACT(13); GP_RHS_EXACT(14); GP_RHS_EXACT(15); GP_RHS_EXACT(16);
#undef GP_RHS_EXACT
        default: return launch_rhs<0>(grid, smem, s, r);
    }
}
static_assert(kPowMaxD == 16, "launch_rhs_exact covers d = 1 .. kPowMaxD");

cudaError_t launch_var_points(const VarCall& c, int m0, int npb, float2* RX, float2* MP, cudaStream_t s,
                              int* kernels) {
    *kernels = 0;
    RhsArgs r;
    r.n = c.n; r.d = c.d; r.nt = c.nt; r.N = c.N; r.m0 = m0;
    r.x = c.x; r.theta = c.theta; r.p = c.p; r.corr = c.corr; r.xs = c.xs; r.w = c.w;
    r.RX = RX;
    r.MP = MP;
    r.tab = c.rtab;
    r.tabpow = !corr_is_matern(c.corr) && pow_mode(c.p) == kPowGeneral && c.d <= kPowMaxD;
    // binomial coefficients C(p, k) of (1 + u)^p
    const double b2 = c.p * (c.p - 1.0) / 2.0, b3 = b2 * (c.p - 2.0) / 3.0, b4 = b3 * (c.p - 3.0) / 4.0;
    r.c2 = b2;
    r.c3 = (float)b3;
    r.c4 = (float)b4;
    r.c5 = (float)(b4 * (c.p - 4.0) / 5.0);
    const size_t rsmem = (size_t)(2 * GP_NB * c.d + c.d + kExpTab) * sizeof(dfl) +
                         (r.tabpow ? (size_t)(c.d * kPowMs + kPowN) * sizeof(dfl) + kPowN * sizeof(float) : 0);
    cudaError_t e = r.tabpow ? launch_rhs_exact(c.d, dim3(c.nt, npb), rsmem, s, r)
                             : launch_rhs<0>(dim3(c.nt, npb), rsmem, s, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_var_mean<<<(npb * GP_NB + 255) / 256, 256, 0, s>>>(MP, c.nt, c.N, m0, npb, c.sc, c.yhat);
    *kernels = 2;
    return cudaGetLastError();
}

size_t var_rhs_tab_bytes() { return ((size_t)kTabLen * sizeof(float2) + 255) & ~(size_t)255; }

// The r kernel's tables (they depend on p alone): 1 kernel.
cudaError_t launch_var_rhs_tables(const VarCall& c, cudaStream_t s, int* kernels) {
    k_var_rhs_tables<<<(kTabInv + kPowN + 255) / 256, 256, 0, s>>>(c.p, c.rtab);
    *kernels = 1;
    return cudaGetLastError();
}

// The tensor-core pass over npb point blocks from point m0, whose r values
// are in RX, on min(npb, grid) CTAs with their slices of V and C_J in VS and
// CS: 1 kernel.
cudaError_t launch_var_pass(const VarCall& c, int m0, int npb, const float2* RX, __nv_bfloat16* VS,
                            __nv_bfloat16* CS, int grid, cudaStream_t s, int* kernels) {
    *kernels = 0;
    if (!var_tc_fits()) return cudaErrorNotSupported;
    VarArgs g;
    g.nt = c.nt; g.npb = npb; g.N = c.N; g.m0 = m0; g.ev = c.ev;
    g.LS = c.t.LS; g.LE = c.t.LE; g.WS = c.t.WS; g.WE = c.t.WE;
    g.a = c.a; g.sc = c.sc; g.c0 = c.c0; g.RX = RX;
    g.VS = VS; g.CS = CS;
    g.vs_stride = (size_t)kVarSlices * 4 * c.nt * kChunkElems;
    g.cs_stride = (size_t)kVarWSlices * 4 * kChunkElems;
    g.s2 = c.s2; g.err = c.err; g.inject_timeout = c.inject_timeout;
    static std::atomic<size_t> tattr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_var_tc, kVarSmem, tattr);
    if (e != cudaSuccess) return e;
    k_var_tc<<<npb < grid ? npb : grid, kVarThreads, kVarSmem, s>>>(g);
    *kernels = 1;
    return cudaGetLastError();
}

}  // namespace gp
