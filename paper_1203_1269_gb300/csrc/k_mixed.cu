// k_mixed.cu -- the split-precision (GP_MIXED) factorisation around its
// tensor-core GEMMs (k_gemm.cu), and the solves.
//
// Blocked right-looking Cholesky of R(theta) + delta I (Section 3 of the
// paper factors R by Cholesky for the determinant and the solves) with the
// off-diagonal work on the tensor cores:
//
//   diag   L_JJ = chol(A_JJ), W_J = L_JJ^-1        double-float (k_diag_mixed)
//   panel  L_IJ = A_IJ W_J^T            I > J      split GEMM (k_gemm.cu)
//   update A_IK -= L_IJ L_KJ^T      J < K <= I     split GEMM (k_gemm.cu)
//
// Split GEMM (after Ozaki, Ogita, Oishi & Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication",
// Numer. Algorithms 59, 2012): each row i of an operand is scaled by 2^(7-E_i)
// (|row| < 2^E_i) and cut into s slices q_a 2^(-8a) with integers |q_a| <= 128,
//     row = 2^(E_i - 7) sum_a q_a 2^(-8a),
// which bf16 holds exactly; this file's slicing kernels write them as the
// pre-swizzled images the MMA descriptors read (mixed_common.cuh).  The
// first forward solve L [x_1 x_y] = [1 Y] is carried out inside the
// factorisation (the diagonal kernel and the slicing of each solved panel).
//
// Solves: the backward substitution with the double-float factor, two
// right-hand sides, then iterative refinement against the double-float copy
// of R (residual r = b - R x, forward correction z = L^-1 r), all
// tile-parallel, with the sums of eq. 3 taken from forward-only identities
// (k_refine_check) and a per-candidate stopping rule; then the profile
// likelihood.
#include "slices.cuh"

namespace gp {

namespace {

// ----------------------------------------------------------- kernels -------

// Diagonal block of column J in double-float on the FP32 pipes (an FP64
// instruction costs about 64 FP32 ones here): L_JJ = chol(A_JJ), log-det,
// the reciprocal diagonal, and W = L_JJ^-1 with the slices of W's rows.
// The block lives in shared memory as a packed lower triangle (row-major,
// P[r(r+1)/2 + c]), 66 KB; two 512-thread CTAs share an SM.
//
// Factor and inverse run in one right-looking sweep over c = 0 .. 127.  At
// step c, position (i, p) of the triangle holds, for rows i > c,
//   p <  c:  acc_ip = sum_{k<c} L_ik W_kp   (the inverse's partial sums)
//   p >= c:  a_ip, the Cholesky trailing matrix,
// and row c holds acc_c. below the diagonal and a_cc on it.  Phase 1 (one
// thread per row p) finishes column c of L (L_pc = a_pc / L_cc, written out)
// and row c of W (W_cp = -acc_cp / L_cc, W_cc = 1 / L_cc), and builds
//   V_p = W_cp (p <= c),   V_p = -L_pc (p > c).
// Phase 2 applies one rank-1 step to every row i > c, a warp per row:
//   X_ip += L_ic V_p for p <= i   (X_ic = L_ic V_c: the first term of acc_ic),
// which is the Cholesky update a_ip -= L_ic L_pc for p > c and the inverse's
// acc_ip += L_ic W_cp for p <= c.  The lane that finishes a_{c+1,c+1} takes
// the next pivot (1 / sqrt from a float seed, refined on the FP32 pipes; see
// take_pivot).
// After step 127 the triangle holds W.
constexpr int kDiagThreads = 512;
constexpr int kPacked = GP_NB * (GP_NB + 1) / 2;

__device__ __forceinline__ int prow(int r) { return r * (r + 1) / 2; }

__global__ void __launch_bounds__(kDiagThreads) k_diag_mixed(MixedBatch b, int J) {
    extern __shared__ dfl P[];             // kPacked double-float values
    __shared__ dfl V[GP_NB];
    __shared__ dfl dinv[GP_NB];            // 1 / L_cc
    __shared__ dfl lcc[GP_NB];             // L_cc
    __shared__ dfl bj[2][GP_NB];
    __shared__ dfl xpart[2][GP_NB];
    __shared__ double lsum[GP_NB / 32];
    __shared__ double psum[GP_NB / 32];
    __shared__ int failed;
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    float2* T = df_tile(b, b.A, t, J, J);
    for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kDiagThreads) {
        const int rr = q & 127, cc = q >> 7;
        if (rr >= cc) cp_async8(P + prow(rr) + cc, T + q);
    }
    if (threadIdx.x == 0) failed = -1;
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kDiagThreads / 32;
    // pivot c: 1 / sqrt(a) from rsqrtf's seed (about 22 correct bits), one
    // float Newton step to y1 (about 24 bits), then y = y1 (1 + e/2 + 3 e^2/8)
    // with e = 1 - a y1^2: Newton's step with its second-order term, the next
    // term (5 e^3 / 16) being below 2^-65.  e is about 2^-23 and needed to
    // float precision only, so it comes from the exact products a.hi y1 and
    // (a.hi y1) y1 (1 - q_h is exact, q_h lying within 2^-22 of 1), and y is
    // the exact sum y1 + corr: about 2^-46 relative, as two double-float
    // Newton steps give, in a quarter of their dependent chain, which matters
    // since the pivot is the sweep's critical path.  Pivots outside
    // [2^-100, 2^100] (the float seed's comfortable range) take the double
    // route.
    auto take_pivot = [&](int c, dfl a) {
        dfl y, l;
        if (!(a.hi > 0.f) || !isfinite(a.hi)) {
            failed = c;
            y = dfl{1.f, 0.f};
            l = y;
        } else if (a.hi > 7.9e-31f && a.hi < 1.26e30f) {
            const float y0 = rsqrtf(a.hi);
            const float p0 = __fmul_rn(a.hi, y0);
            const float y1 = __fmaf_rn(__fmul_rn(y0, 0.5f), __fmaf_rn(-p0, y0, 1.f), y0);
            const float ph = __fmul_rn(a.hi, y1);
            const float pl = __fmaf_rn(a.hi, y1, -ph);
            const float qh = __fmul_rn(ph, y1);
            const float ql = __fmaf_rn(pl, y1, __fmaf_rn(ph, y1, -qh));
            const float rl = __fmul_rn(__fmul_rn(a.lo, y1), y1);
            const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, qh), ql), rl);
            const float h = __fmul_rn(y1, 0.5f);
            const float corr = __fmaf_rn(h, e, __fmul_rn(__fmul_rn(h, __fmul_rn(e, e)), 0.75f));
            fast_two_sum(y1, corr, y.hi, y.lo);
            l = df_mul(a, y);
        } else {
            const double piv = df_to_double(a);
            const double ld = sqrt(piv);
            y = df_from_double(1.0 / ld);
            l = df_from_double(ld);
        }
        lcc[c] = l;
        dinv[c] = y;
    };
    if (threadIdx.x == 0) take_pivot(0, P[0]);
    __syncthreads();
    for (int c = 0; c < GP_NB; ++c) {
        if (failed >= 0) break;            // read after a barrier: uniform
        // phase 1: column c of L (out), row c of W, V
        if (threadIdx.x < GP_NB) {
            const int p = threadIdx.x;
            const dfl di = dinv[c];
            if (p < c) {
                const dfl w = df_neg(df_mul(di, P[prow(c) + p]));
                P[prow(c) + p] = w;
                V[p] = w;
            } else if (p == c) {
                df_store(T + (size_t)c * GP_NB + c, lcc[c]);
                P[prow(c) + c] = di;
                V[c] = di;
            } else {
                const dfl l = df_mul(P[prow(p) + c], di);
                df_store(T + (size_t)c * GP_NB + p, l);
                V[p] = df_neg(l);
                P[prow(p) + c] = dfl{0.f, 0.f};   // restarts in phase 2 as acc_pc = L_pc V_c
            }
        }
        __syncthreads();
        if (c + 1 == GP_NB) break;
        // phase 2: rows i > c, X_ip += L_ic V_p (p <= i), a warp per row; warp
        // 0 takes only row c + 1 and its pivot, the others deal the rest two
        // rows at a time (both rows' loads first: eight independent
        // multiply-adds per lane).  A row i reaches only the 32-column blocks
        // j <= i / 32, a test that is uniform across the warp.
        dfl vl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) vl[j] = V[lane + 32 * j];
        if (warp == 0) {
            const int i = c + 1;
            const dfl m = df_neg(V[i]);    // L_ic
            dfl* row = P + prow(i);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = lane + 32 * j;
                if (32 * j <= i && p <= i) {
                    const dfl x0 = row[p];
                    const dfl x = df_fma(m, vl[j], x0);
                    if (p == c + 1)
                        take_pivot(c + 1, x);
                    else
                        row[p] = x;
                }
            }
        } else {
            constexpr int kRowStep = kWarps - 1;
            for (int i = c + 1 + warp; i < GP_NB; i += 2 * kRowStep) {
                const int i2 = i + kRowStep;
                const bool two = i2 < GP_NB;
                const dfl m1 = df_neg(V[i]);
                const dfl m2 = two ? df_neg(V[i2]) : dfl{0.f, 0.f};
                dfl* r1 = P + prow(i);
                dfl* r2 = P + prow(two ? i2 : i);
                dfl x1[4], x2[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = lane + 32 * j;
                    if (32 * j <= i) x1[j] = (p <= i) ? r1[p] : dfl{0.f, 0.f};
                    if (two && 32 * j <= i2) x2[j] = (p <= i2) ? r2[p] : dfl{0.f, 0.f};
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = lane + 32 * j;
                    if (32 * j <= i && p <= i) r1[p] = df_fma(m1, vl[j], x1[j]);
                    if (two && 32 * j <= i2 && p <= i2) r2[p] = df_fma(m2, vl[j], x2[j]);
                }
            }
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
    // log-det: sum of log L_cc over the block in a fixed order (warp trees,
    // then the four warp sums in turn); reciprocal diagonal out
    // and the sum of 1 / L_cc^2 over the block's real rows (the refinement's
    // estimate of the log-det's own error, k_refine_check)
    if (threadIdx.x < GP_NB) {
        double v = log(df_to_double(lcc[threadIdx.x]));
        const double di = df_to_double(dinv[threadIdx.x]);
        double q = (J * GP_NB + (int)threadIdx.x < b.n) ? di * di : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, o);
            q += __shfl_down_sync(0xffffffffu, q, o);
        }
        if (lane == 0) {
            lsum[warp] = v;
            psum[warp] = q;
        }
        float2* rinv = b.Z + (size_t)t * b.z_stride + (size_t)4 * b.nt * GP_NB + J * GP_NB;
        df_store(rinv + threadIdx.x, dinv[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ld = 0.0, pq = 0.0;
        for (int w = 0; w < GP_NB / 32; ++w) {
            ld += lsum[w];
            pq += psum[w];
        }
        b.st[t].logdet += 2.0 * ld;
        b.st[t].piv_inv += pq;
    }
    // W as a double-float tile (column-major, zeros above the diagonal) for
    // the diagonal-block products of the solves
    // and row-major (W^T column-major) for the backward substitution
    {
        float2* Wt = b.WT + (size_t)t * b.wt_stride + (size_t)J * GP_TILE_ELEMS;
        float2* Wr = b.WR + (size_t)t * b.wt_stride + (size_t)J * GP_TILE_ELEMS;
        for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kDiagThreads) {
            const int rr = q & 127, cc = q >> 7;
            Wt[q] = (rr >= cc) ? make_float2(P[prow(rr) + cc].hi, P[prow(rr) + cc].lo) : make_float2(0.f, 0.f);
            // row cc, column rr of W
            Wr[q] = (cc >= rr) ? make_float2(P[prow(cc) + rr].hi, P[prow(cc) + rr].lo) : make_float2(0.f, 0.f);
        }
    }
    // row c of W: exponent (of the largest high word, as the panel slicing
    // takes it) and slices; one warp per row, all on the FP32 pipes
    __nv_bfloat16* WS = b.WS + (size_t)t * b.ws_stride;
    int* WE = b.WE + (size_t)t * b.we_stride;
    for (int c = warp; c < GP_NB; c += kWarps) {
        const dfl* w = P + prow(c);
        float mx = 0.f;
        for (int k = lane; k <= c; k += 32) mx = fmaxf(mx, fabsf(w[k].hi));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int E = exponent_of(mx);
        if (lane == 0) WE[c] = E;
        // x 2^(7 - E) exactly (two factors when 7 - E leaves the float range)
        const int e2 = 7 - E;
        const int ea = e2 > 127 ? 127 : (e2 < -126 ? -126 : e2);
        const int eb = e2 - ea;
        const float sa = __int_as_float((ea + 127) << 23);
        const float sb = (eb == 0) ? 1.f : __int_as_float(((eb > 127 ? 127 : (eb < -126 ? -126 : eb)) + 127) << 23);
        // lane handles columns 4*lane .. 4*lane+3 (half of one 16-byte piece)
        const int k0 = 4 * lane;
        float m[4][GP_MAX_SLICES];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const dfl x = (k0 + e <= c) ? w[k0 + e] : dfl{0.f, 0.f};
            cut_slices(__fmul_rn(__fmul_rn(x.hi, sa), sb), __fmul_rn(__fmul_rn(x.lo, sa), sb), b.ps, m[e]);
        }
        const uint32_t off = image_piece(c, k0 & ~7) + ((k0 & 4) ? 8u : 0u);
#pragma unroll
        for (int a = 0; a < GP_MAX_SLICES; ++a) {
            if (a >= b.ps) break;
            uint2 v;
            v.x = pack_bf16x2(m[0][a], m[1][a]);
            v.y = pack_bf16x2(m[2][a], m[3][a]);
            uint8_t* dst = reinterpret_cast<uint8_t*>(WS + (size_t)(a * kChunks + (k0 >> 5)) * kChunkElems);
            *reinterpret_cast<uint2*>(dst + off) = v;
        }
    }
    if (b.fwd) {
        // forward solve, block J: x_J = W (b_J - sum_{K<J} L_JK x_K), the sum
        // already subtracted by the slicing of panels K < J; b_J in, x_J out
        // (Z columns 0, 1), in double-float: thread (k, r, h) sums the
        // columns c = h, h + 2, ... of row r, then the two halves add in a
        // fixed order
        float2* zJ = b.Z + (size_t)t * b.z_stride + (size_t)J * GP_NB;
        const int k = (threadIdx.x >> 7) & 1, r = threadIdx.x & 127, h = threadIdx.x >> 8;
        float2* zk = zJ + (size_t)k * b.nt * GP_NB;
        if (threadIdx.x < 2 * GP_NB) bj[k][r] = df_load(zk + r);
        __syncthreads();
        const dfl* w = P + prow(r);
        dfl sum = {0.f, 0.f};
        for (int c = h; c <= r; c += 2) sum = df_fma(w[c], bj[k][c], sum);
        if (h == 1) xpart[k][r] = sum;
        __syncthreads();
        if (h == 0) df_store(zk + r, df_add(sum, xpart[k][r]));
    }
}

// Slices of the panel tiles (I, J), I = J + 1 + blockIdx.x / 2, into row
// block I of PS.  A CTA of 512 threads takes one half (64 rows) of a tile:
// thread (r, q, u) owns row r's columns 32q + 16u .. 32q + 16u + 15, two of
// the 16-byte pieces of image chunk q, so it loads its values once
// (coalesced along r) and writes only its own pieces; 16 values per thread
// leave registers for four CTAs per SM, whose loads overlap each other's
// slicing.  The eight owners of a row agree on the row's exponent through
// shared memory.
constexpr int kSplitThreads = 512;
constexpr int kSplitParts = 8;                          // column parts of a row
constexpr int kSplitRows = kSplitThreads / kSplitParts; // rows of a tile per CTA
constexpr int kSplitCols = GP_NB / kSplitParts;         // 16 columns per thread
// k_split_fused: 16 columns of one of the two panels per thread, a quarter tile
constexpr int kFusedParts = 16;
constexpr int kFusedRows = kSplitThreads / kFusedParts;

// gemv (with b.fwd; the slicing of the solved panel for the update): the
// forward solve's panel step b_I -= L_IJ x_J for this CTA's rows, two
// right-hand sides, from the values already in registers.  c0: the first of
// the thread's 16 columns.
template <int NC, int ROWS>
__device__ __forceinline__ void fwd_partials(const float2 (&v)[NC], const dfl (*xs)[GP_NB], int c0,
                                             int part, int rl, dfl (*red)[2][ROWS]) {
    dfl p0 = {0.f, 0.f}, p1 = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const dfl l = {v[j].x, v[j].y};
        p0 = df_fma(l, xs[0][c0 + j], p0);
        p1 = df_fma(l, xs[1][c0 + j], p1);
    }
    red[part][0][rl] = p0;
    red[part][1][rl] = p1;
}

// b_I[r] -= the PARTS column parts' partial sums, pairwise in a fixed order
// (parts 0 and 1 take one right-hand side each); after a barrier that
// follows fwd_partials
template <int PARTS, int ROWS>
__device__ __forceinline__ void fwd_apply(const MixedBatch& b, int t, int I, int r, int part, int rl,
                                          const dfl (*red)[2][ROWS]) {
    if (part < 2) {
        const int k = part;
        dfl acc[PARTS];
#pragma unroll
        for (int i = 0; i < PARTS; ++i) acc[i] = red[i][k][rl];
#pragma unroll
        for (int w = 1; w < PARTS; w *= 2)
#pragma unroll
            for (int i = 0; i + w < PARTS; i += 2 * w) acc[i] = df_add(acc[i], acc[i + w]);
        float2* z = b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB + (size_t)I * GP_NB + r;
        df_store(z, df_sub(df_load(z), acc[0]));
    }
}

__global__ void __launch_bounds__(kSplitThreads) k_split_panel(MixedBatch b, int J, int ns, int gemv) {
    __shared__ float pmax[kSplitParts][kSplitRows];
    __shared__ dfl xs[2][GP_NB];
    __shared__ dfl red[kSplitParts][2][kSplitRows];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int I = J + 1 + blockIdx.x / 2;
    const float2* src = df_tile(b, b.A, t, I, J);
    const int rl = threadIdx.x % kSplitRows, part = threadIdx.x / kSplitRows;
    const int q = part >> 1, u = part & 1, c0 = kSplitCols * part;
    const int r = (blockIdx.x & 1) * kSplitRows + rl;
    gemv = gemv && b.fwd;
    if (gemv && threadIdx.x < 2 * GP_NB) {
        // x_J of both right-hand sides
        const int k = threadIdx.x >> 7, c = threadIdx.x & 127;
        xs[k][c] = df_load(b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB + (size_t)J * GP_NB + c);
    }
    float2 v[kSplitCols];
#pragma unroll
    for (int j = 0; j < kSplitCols; ++j) v[j] = src[(size_t)(c0 + j) * GP_NB + r];
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < kSplitCols; ++j) mx = fmaxf(mx, fabsf(v[j].x));
    pmax[part][rl] = mx;
    __syncthreads();
    if (gemv) fwd_partials(v, xs, c0, part, rl, red);
#pragma unroll
    for (int k = 0; k < kSplitParts; ++k) mx = fmaxf(mx, pmax[k][rl]);
    const int E = exponent_of(mx);
    if (part == 0) pe_block(b, t, I)[r] = E;
    float sa, sb;
    slice_scale(E, sa, sb);
    uint8_t* chunk0 = reinterpret_cast<uint8_t*>(ps_block(b, t, I) + (size_t)q * kChunkElems);
    slice_pieces(v, sa, sb, r, 16 * u, ns, chunk0, (size_t)kChunks * kChunkBytes);
    if (gemv) {
        __syncthreads();
        fwd_apply<kSplitParts>(b, t, I, r, part, rl, red);
    }
}

// Slices of two adjacent panels at once, for the fused (K = 256) trailing
// update: row r of row block I = J + 2 + blockIdx.x / 4 spans tiles (I, J) and
// (I, J + 1) and gets one exponent for all 256 columns, so the products of
// both panels accumulate in the same tensor-memory groups.  A CTA takes a
// quarter tile (32 rows); thread (r, part) owns 16 columns of one panel
// (parts 0-7 panel J, 8-15 panel J + 1; the same two pieces of an image
// chunk as in k_split_panel), so every tile is read once and every slice
// written in 32-byte stores; the row maximum spans all 16 parts.
__global__ void __launch_bounds__(kSplitThreads) k_split_fused(MixedBatch b, int J) {
    __shared__ float pmax[kFusedParts][kFusedRows];
    __shared__ dfl xs[2][GP_NB];
    __shared__ dfl red[kFusedParts / 2][2][kFusedRows];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int I = J + 2 + blockIdx.x / 4;
    const int rl = threadIdx.x % kFusedRows, part = threadIdx.x / kFusedRows;
    const int panel = part >> 3, lp = part & 7;
    const int q = lp >> 1, u = lp & 1, c0 = kSplitCols * lp;
    const int r = (blockIdx.x & 3) * kFusedRows + rl;
    if (b.fwd && threadIdx.x < 2 * GP_NB) {
        // x_{J+1}: the panel J term was applied by k_split_panel
        const int k = threadIdx.x >> 7, c = threadIdx.x & 127;
        xs[k][c] = df_load(b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB + (size_t)(J + 1) * GP_NB + c);
    }
    const float2* src = df_tile(b, b.A, t, I, J + panel);
    float2 v[kSplitCols];
#pragma unroll
    for (int j = 0; j < kSplitCols; ++j) v[j] = src[(size_t)(c0 + j) * GP_NB + r];
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < kSplitCols; ++j) mx = fmaxf(mx, fabsf(v[j].x));
    pmax[part][rl] = mx;
    __syncthreads();
    if (b.fwd && panel == 1) fwd_partials(v, xs, c0, lp, rl, red);
#pragma unroll
    for (int k = 0; k < kFusedParts; ++k) mx = fmaxf(mx, pmax[k][rl]);
    const int E = exponent_of(mx);
    if (part == 0) fe_block(b, t, I)[r] = E;
    float sa, sb;
    slice_scale(E, sa, sb);
    const size_t slice_bytes = (size_t)2 * kChunks * kChunkBytes;
    uint8_t* base = reinterpret_cast<uint8_t*>(pf_block(b, t, I));
    slice_pieces(v, sa, sb, r, 16 * u, b.s, base + (size_t)(4 * panel + q) * kChunkElems * 2, slice_bytes);
    if (b.fwd) {
        __syncthreads();
        fwd_apply<kFusedParts / 2>(b, t, I, r, part, rl, red);
    }
}

// ------------------------------------------------------------ solves -------
// Z (per instance, float2): column k of length npad at Z + k * npad.
//   0: x_1   1: x_y   2, 3: residual / correction   4: 1 / L_ii
// The substitutions and the residual are tile-parallel (kernels below);
// tiles whose transpose is needed are staged in shared memory column by
// column with one entry of padding, so that a thread walking a column and
// one walking a row both read conflict-free (2-way for the 8-byte entries).

constexpr int kSolveThreads = 512;   // the finalising reduction
constexpr int kTs = GP_NB + 1;       // staged column stride of a 128-row tile part

__device__ __forceinline__ float2* zcol(const MixedBatch& b, int t, int k) {
    return b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB;
}

// Fixed-order sum over the block of a double-float value held per thread.
__device__ dfl block_sum_df(dfl v, dfl* red) {
    for (int o = 16; o > 0; o >>= 1) {
        dfl w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        dfl s = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s = df_add(s, red[i]);
        red[0] = s;
    }
    __syncthreads();
    dfl s = red[0];
    __syncthreads();
    return s;
}


// [1 Y] (zero on padded rows) into Z columns 0, 1: the right-hand sides of
// the forward solve that the factorisation carries out block by block
__global__ void k_rhs_init(MixedBatch b) {
    const int t = blockIdx.y;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= b.nt * GP_NB) return;
    const bool in = gi < b.n;
    df_store(zcol(b, t, 0) + gi, dfl{in ? 1.f : 0.f, 0.f});
    df_store(zcol(b, t, 1) + gi, in ? df_from_double(b.y[gi]) : dfl{0.f, 0.f});
}




// Forward and backward substitution with the double-float factor for two
// columns (c0, c0 + 1) of Z in place, tile-parallel: block column by block
// column, a small kernel finishes the diagonal block from the partial
// products of the tiles already applied (fixed order), and a tile kernel
// forms the next partial products of every tile of that block column (or
// row) at once, one CTA per tile half.  Partial products live in RP:
// per lower tile q, [2 halves][2 columns][128] double-float values.
constexpr int kSubThreads = 256;

__device__ __forceinline__ bool sub_active(const MixedBatch& b, int t) {
    return b.st[t].status == GP_OK && !b.st[t].hager_done && !b.st[t].refine_done;
}

__device__ __forceinline__ float2* rp_part(const MixedBatch& b, int t, int I, int J) {
    return b.RP + (size_t)t * b.rp_stride + (size_t)tile_index(I, J, b.nt) * kRpTile;
}

__device__ __forceinline__ dfl df_load_cg(const float2* p) {
    const float2 v = __ldcg(p);
    return {v.x, v.y};
}

// The diagonal steps run either as their own launch (the first block of a
// pass) or inside the tile launch before them, by whichever of the two CTAs
// writing the block's last partial products finishes second: each of them
// fences its partial products device-wide and counts itself on the block's
// counter (zeroed per pass); the second reads all the block's partial
// products in the same fixed order as a separate launch would.  No CTA
// waits for another.
__device__ __forceinline__ bool second_of_two(const MixedBatch& b, int t, int blk) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(b.SC + (size_t)t * b.sc_stride + blk, 1) == 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// forward, block J: z_J <- W_J (z_J - sum_{K<J} L_JK z_K), W_J = L_JJ^-1.
// Thread (r, h) takes both right-hand sides of row r over half h of the
// terms (every other partial-product tile, then columns 64h .. 64h + 63 of
// the column-major WT, one load serving both sums); the halves add in a
// fixed order.  part: 2 x 2 x 128 scratch.
__device__ __forceinline__ void fwd_diag_step(const MixedBatch& b, int t, int c0, int J, dfl (*rhs)[GP_NB],
                                              dfl (*part)[2][GP_NB]) {
    const int r = threadIdx.x & 127, h = threadIdx.x >> 7;
    float2* z0 = zcol(b, t, c0) + (size_t)J * GP_NB;
    float2* z1 = zcol(b, t, c0 + 1) + (size_t)J * GP_NB;
    dfl p0 = {0.f, 0.f}, p1 = {0.f, 0.f};
#pragma unroll 4
    for (int K = h; K < J; K += 2) {
        const float2* pp = rp_part(b, t, J, K) + r;
        p0 = df_add(p0, df_add(df_load_cg(pp), df_load_cg(pp + 2 * GP_NB)));
        p1 = df_add(p1, df_add(df_load_cg(pp + GP_NB), df_load_cg(pp + 3 * GP_NB)));
    }
    part[h][0][r] = p0;
    part[h][1][r] = p1;
    __syncthreads();
    if (h == 0) {
        rhs[0][r] = df_sub(df_load(z0 + r), df_add(part[0][0][r], part[1][0][r]));
        rhs[1][r] = df_sub(df_load(z1 + r), df_add(part[0][1][r], part[1][1][r]));
    }
    __syncthreads();
    // 64 columns (W is zero above its diagonal: a fixed trip count lets the
    // loads run ahead of the accumulation chains)
    const float2* W = b.WT + (size_t)t * b.wt_stride + (size_t)J * GP_TILE_ELEMS;
    dfl a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, b0 = {0.f, 0.f}, b1 = {0.f, 0.f};
#pragma unroll 16
    for (int c = 64 * h; c < 64 * h + 64; c += 2) {
        const dfl w0 = df_load(W + (size_t)c * GP_NB + r), w1 = df_load(W + (size_t)(c + 1) * GP_NB + r);
        a0 = df_fma(w0, rhs[0][c], a0);
        b0 = df_fma(w0, rhs[1][c], b0);
        a1 = df_fma(w1, rhs[0][c + 1], a1);
        b1 = df_fma(w1, rhs[1][c + 1], b1);
    }
    __syncthreads();
    part[h][0][r] = df_add(a0, a1);
    part[h][1][r] = df_add(b0, b1);
    __syncthreads();
    if (h == 0) {
        df_store(z0 + r, df_add(part[0][0][r], part[1][0][r]));
        df_store(z1 + r, df_add(part[0][1][r], part[1][1][r]));
    }
}

__global__ void __launch_bounds__(kSubThreads) k_fwd_diag(MixedBatch b, int c0, int J) {
    __shared__ dfl rhs[2][GP_NB];
    __shared__ dfl part[2][2][GP_NB];
    const int t = blockIdx.x;
    if (!sub_active(b, t)) return;
    fwd_diag_step(b, t, c0, J, rhs, part);
}

// forward, tiles (I, J), I > J, half h of the columns: L_IJ(:, h) z_J(h);
// the CTA finishing tile (J + 1, J) second then takes block J + 1's
// diagonal step
__global__ void __launch_bounds__(kSubThreads) k_fwd_tiles(MixedBatch b, int c0, int J) {
    __shared__ dfl xs[2][GP_NB / 2];
    __shared__ dfl part[2][2][GP_NB];
    __shared__ dfl rhs[2][GP_NB];
    const int t = blockIdx.y;
    if (!sub_active(b, t)) return;
    const int I = J + 1 + (blockIdx.x >> 1), h = blockIdx.x & 1;
    const int tid = threadIdx.x;
    // W_{J+1} heads for L2 for the diagonal step
    if (tid == 0 && I == J + 1 && h == 0)
        prefetch_l2(b.WT + (size_t)t * b.wt_stride + (size_t)(J + 1) * GP_TILE_ELEMS, GP_TILE_ELEMS * sizeof(float2));
    if (tid < GP_NB) xs[tid >> 6][tid & 63] = df_load(zcol(b, t, c0 + (tid >> 6)) + (size_t)J * GP_NB + 64 * h + (tid & 63));
    __syncthreads();
    const float2* L = df_tile(b, b.A, t, I, J) + (size_t)h * 64 * GP_NB;
    const int r = tid & 127, g = tid >> 7;
    dfl u0 = {0.f, 0.f}, u1 = {0.f, 0.f};
#pragma unroll 8
    for (int c = 32 * g; c < 32 * g + 32; ++c) {
        const float2 l = __ldg(L + (size_t)c * GP_NB + r);
        const dfl ld = {l.x, l.y};
        u0 = df_fma(ld, xs[0][c], u0);
        u1 = df_fma(ld, xs[1][c], u1);
    }
    part[g][0][r] = u0;
    part[g][1][r] = u1;
    __syncthreads();
    const int k = tid >> 7;
    df_store(rp_part(b, t, I, J) + (h * 2 + k) * GP_NB + r, df_add(part[0][k][r], part[1][k][r]));
    if (I == J + 1 && second_of_two(b, t, I)) fwd_diag_step(b, t, c0, I, rhs, part);
}

// backward, block K: z_K <- W_K^T (z_K - sum_{K' > K} L_K'K^T z_K'); W^T
// from the row-major copy WR (thread (c, h) reads column c of W along rows
// 64h .. 64h + 63, both right-hand sides per load; the partial-product
// tiles alternate between the halves); the halves add in a fixed order.
// With add_to >= 0 the result is also added into (add_to, add_to + 1).
__device__ __forceinline__ void bwd_diag_step(const MixedBatch& b, int t, int c0, int K, int add_to,
                                              dfl (*rhs)[GP_NB], dfl (*part)[2][GP_NB]) {
    const int nt = b.nt;
    const int c = threadIdx.x & 127, h = threadIdx.x >> 7;
    float2* z0 = zcol(b, t, c0) + (size_t)K * GP_NB;
    float2* z1 = zcol(b, t, c0 + 1) + (size_t)K * GP_NB;
    dfl p0 = {0.f, 0.f}, p1 = {0.f, 0.f};
#pragma unroll 4
    for (int K2 = K + 1 + h; K2 < nt; K2 += 2) {
        const float2* pp = rp_part(b, t, K2, K) + c;
        p0 = df_add(p0, df_add(df_load_cg(pp), df_load_cg(pp + 2 * GP_NB)));
        p1 = df_add(p1, df_add(df_load_cg(pp + GP_NB), df_load_cg(pp + 3 * GP_NB)));
    }
    part[h][0][c] = p0;
    part[h][1][c] = p1;
    __syncthreads();
    if (h == 0) {
        rhs[0][c] = df_sub(df_load(z0 + c), df_add(part[0][0][c], part[1][0][c]));
        rhs[1][c] = df_sub(df_load(z1 + c), df_add(part[0][1][c], part[1][1][c]));
    }
    __syncthreads();
    const float2* Wr = b.WR + (size_t)t * b.wt_stride + (size_t)K * GP_TILE_ELEMS;
    dfl a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, b0 = {0.f, 0.f}, b1 = {0.f, 0.f};
#pragma unroll 16
    for (int r = 64 * h; r < 64 * h + 64; r += 2) {
        const dfl w0 = df_load(Wr + (size_t)r * GP_NB + c), w1 = df_load(Wr + (size_t)(r + 1) * GP_NB + c);
        a0 = df_fma(w0, rhs[0][r], a0);
        b0 = df_fma(w0, rhs[1][r], b0);
        a1 = df_fma(w1, rhs[0][r + 1], a1);
        b1 = df_fma(w1, rhs[1][r + 1], b1);
    }
    __syncthreads();
    part[h][0][c] = df_add(a0, a1);
    part[h][1][c] = df_add(b0, b1);
    __syncthreads();
    if (h == 0) {
        const dfl x0 = df_add(part[0][0][c], part[1][0][c]);
        const dfl x1 = df_add(part[0][1][c], part[1][1][c]);
        df_store(z0 + c, x0);
        df_store(z1 + c, x1);
        if (add_to >= 0) {
            float2* acc0 = zcol(b, t, add_to) + (size_t)K * GP_NB + c;
            float2* acc1 = zcol(b, t, add_to + 1) + (size_t)K * GP_NB + c;
            df_store(acc0, df_add(df_load(acc0), x0));
            df_store(acc1, df_add(df_load(acc1), x1));
        }
    }
}

__global__ void __launch_bounds__(kSubThreads) k_bwd_diag(MixedBatch b, int c0, int K, int add_to) {
    __shared__ dfl rhs[2][GP_NB];
    __shared__ dfl part[2][2][GP_NB];
    const int t = blockIdx.x;
    if (!sub_active(b, t)) return;
    bwd_diag_step(b, t, c0, K, add_to, rhs, part);
}

// backward, tiles (K, I), I < K, half h of the rows: L_KI(h, :)^T z_K(h);
// the half tile is staged column by column (64 rows + 1 of padding) so that
// thread c walks column c conflict-free; the CTA finishing tile (K, K - 1)
// second then takes block K - 1's diagonal step
constexpr int kBwdTs = GP_NB / 2 + 1;
__global__ void __launch_bounds__(kSubThreads) k_bwd_tiles(MixedBatch b, int c0, int K, int add_to) {
    extern __shared__ dfl T[];                  // GP_NB x kBwdTs
    __shared__ dfl xs[2][GP_NB / 2];
    __shared__ dfl part[2][2][GP_NB];
    __shared__ dfl rhs[2][GP_NB];
    const int t = blockIdx.y;
    if (!sub_active(b, t)) return;
    const int I = blockIdx.x >> 1, h = blockIdx.x & 1;
    const int tid = threadIdx.x;
    // W_{K-1} (row-major) heads for L2 for the next diagonal step
    if (tid == 0 && I == K - 1 && h == 0)
        prefetch_l2(b.WR + (size_t)t * b.wt_stride + (size_t)(K - 1) * GP_TILE_ELEMS, GP_TILE_ELEMS * sizeof(float2));
    if (tid < GP_NB) xs[tid >> 6][tid & 63] = df_load(zcol(b, t, c0 + (tid >> 6)) + (size_t)K * GP_NB + 64 * h + (tid & 63));
    const float2* L = df_tile(b, b.A, t, K, I) + 64 * h;
#pragma unroll
    for (int e = tid; e < 64 * GP_NB; e += kSubThreads) {
        const int c = e >> 6, rr = e & 63;
        cp_async8(T + c * kBwdTs + rr, L + (size_t)c * GP_NB + rr);
    }
    cp_async_wait_all();
    __syncthreads();
    const int c = tid & 127, g = tid >> 7;
    const dfl* col = T + c * kBwdTs;
    dfl s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll 8
    for (int rr = 32 * g; rr < 32 * g + 32; ++rr) {
        s0 = df_fma(col[rr], xs[0][rr], s0);
        s1 = df_fma(col[rr], xs[1][rr], s1);
    }
    part[g][0][c] = s0;
    part[g][1][c] = s1;
    __syncthreads();
    const int k = tid >> 7;
    df_store(rp_part(b, t, K, I) + (h * 2 + k) * GP_NB + c, df_add(part[0][k][c], part[1][k][c]));
    // the CTA finishing tile (K, K - 1) second takes block K - 1's diagonal step
    if (I == K - 1 && second_of_two(b, t, I)) bwd_diag_step(b, t, c0, I, add_to, rhs, part);
}

// Residual r = b - R x of the solution columns (0, 1) into columns (2, 3),
// against the double-float copy of R, tile-parallel: one CTA per (lower tile
// (I, J) of the R copy, column half hc) stages its 128 x 64 part and writes
// the partial sums
//   U = R_IJ(:, half) x_J(half)        two columns of 128 (row products)
//   V = R_IJ(:, half)^T x_I            two columns of 64 (column products, I != J)
// into RP; k_resid_reduce adds them per row block in a fixed order.  The
// diagonal tiles of the R copy hold both triangles, so they give U only.
// RP per tile q: U[hc][k][128] then V[hc][k][64] (kRpTile values).
constexpr int kResThreads = 256;
constexpr int kResCols = GP_NB / 2;
static_assert(kRpTile == 2 * 2 * GP_NB + 2 * 2 * kResCols, "residual partial layout");

__global__ void __launch_bounds__(kResThreads) k_resid_tiles(MixedBatch b) {
    extern __shared__ dfl T[];                  // kResCols x kTs
    __shared__ dfl xa[2][kResCols];             // x_J on this half's columns
    __shared__ dfl xb[2][GP_NB];                // x_I
    __shared__ dfl part[2 * 2 * GP_NB];           // U: [2][2][128], then V: [4][2][64]
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK || b.st[t].refine_done) return;
    const int nt = b.nt;
    const int q = blockIdx.x >> 1, hc = blockIdx.x & 1;
    int J = 0, rem = q;
    while (rem >= nt - J) {
        rem -= nt - J;
        ++J;
    }
    const int I = J + rem;
    const int tid = threadIdx.x;
    if (tid < 2 * kResCols) xa[tid >> 6][tid & 63] = df_load(zcol(b, t, tid >> 6) + J * GP_NB + hc * kResCols + (tid & 63));
    xb[tid >> 7][tid & 127] = df_load(zcol(b, t, tid >> 7) + I * GP_NB + (tid & 127));
    const float2* src = df_tile(b, b.Rc, t, I, J) + (size_t)hc * kResCols * GP_NB;
#pragma unroll
    for (int e = tid; e < kResCols * GP_NB; e += kResThreads) cp_async8(T + (e >> 7) * kTs + (e & 127), src + e);
    cp_async_wait_all();
    __syncthreads();
    float2* rp = b.RP + (size_t)t * b.rp_stride + (size_t)q * kRpTile;
    {
        // U: thread (r, h) takes the columns 32h .. 32h + 31 of the half
        const int r = tid & 127, h = tid >> 7;
        dfl u0 = {0.f, 0.f}, u1 = {0.f, 0.f};
#pragma unroll 4
        for (int c = 32 * h; c < 32 * h + 32; ++c) {
            const dfl v = T[c * kTs + r];
            u0 = df_fma(v, xa[0][c], u0);
            u1 = df_fma(v, xa[1][c], u1);
        }
        part[(h * 2 + 0) * GP_NB + r] = u0;
        part[(h * 2 + 1) * GP_NB + r] = u1;
    }
    __syncthreads();
    {
        const int k = tid >> 7, r = tid & 127;
        df_store(rp + (hc * 2 + k) * GP_NB + r, df_add(part[k * GP_NB + r], part[(2 + k) * GP_NB + r]));
    }
    if (I == J) return;                         // uniform
    __syncthreads();
    {
        // V: thread (c, h) takes the rows 32h .. 32h + 31 of column c
        const int c = tid & 63, h = tid >> 6;
        const dfl* col = T + c * kTs;
        dfl s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll 4
        for (int r = 32 * h; r < 32 * h + 32; ++r) {
            s0 = df_fma(col[r], xb[0][r], s0);
            s1 = df_fma(col[r], xb[1][r], s1);
        }
        part[(h * 2 + 0) * kResCols + c] = s0;
        part[(h * 2 + 1) * kResCols + c] = s1;
    }
    __syncthreads();
    if (tid < 2 * kResCols) {
        const int k = tid >> 6, c = tid & 63;
        const dfl v = df_add(df_add(part[(0 + k) * kResCols + c], part[(2 + k) * kResCols + c]),
                             df_add(part[(4 + k) * kResCols + c], part[(6 + k) * kResCols + c]));
        df_store(rp + 4 * GP_NB + (hc * 2 + k) * kResCols + c, v);
    }
}

// r_I = b_I - (sum_{J <= I} U(I, J) + sum_{J > I} V(J, I)) for both columns,
// into Z columns 2, 3; padded rows: R is the identity there and x is zero,
// so r = 0.  One CTA per (row block I, instance).
__global__ void __launch_bounds__(kResThreads) k_resid_reduce(MixedBatch b) {
    const int t = blockIdx.y, I = blockIdx.x;
    if (b.st[t].status != GP_OK || b.st[t].refine_done) return;
    const int nt = b.nt, n = b.n;
    const int k = threadIdx.x >> 7, r = threadIdx.x & 127;
    const float2* rp = b.RP + (size_t)t * b.rp_stride;
    dfl y = {0.f, 0.f};
    for (int J = 0; J <= I; ++J) {
        const float2* u = rp + (size_t)tile_index(I, J, nt) * kRpTile;
        y = df_add(y, df_load(u + k * GP_NB + r));
        y = df_add(y, df_load(u + (2 + k) * GP_NB + r));
    }
    for (int K = I + 1; K < nt; ++K) {
        const float2* v = rp + (size_t)tile_index(K, I, nt) * kRpTile + 4 * GP_NB;
        y = df_add(y, df_load(v + ((r >> 6) * 2 + k) * kResCols + (r & 63)));
    }
    const int gi = I * GP_NB + r;
    dfl bq = {0.f, 0.f};
    if (gi < n) bq = k ? df_from_double(b.y[gi]) : dfl{1.f, 0.f};
    df_store(zcol(b, t, 2 + k) + gi, (gi < n) ? df_sub(bq, y) : dfl{0.f, 0.f});
}

// a = L^-1 1 and b = L^-1 Y (Z columns 0, 1 after the forward solve) into
// columns 8, 9, where the refinement's sums read them
__global__ void k_keep_forward(MixedBatch b) {
    const int t = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int npad = b.nt * GP_NB;
    if (b.st[t].status != GP_OK || i >= 2 * npad) return;
    const int k = i / npad, r = i - k * npad;
    zcol(b, t, 8 + k)[r] = zcol(b, t, k)[r];
}

// The sums of eq. 3 after refinement step `step` (0: the first solve, before
// any correction), and whether the candidate refines further.
//
// With the factor L (L L' ~ R), x = [x_1 x_y] the current solution of
// R x = [1 Y], r = [1 Y] - R x its residual and z = L^-1 r (Z columns 2, 3),
// the refined solution is x + L^-T z, and every sum eq. 3 needs follows
// without that backward substitution, since v' L^-T z = (L^-1 v)' z:
//   1'R^-1 1 = 1'x_1 + a'z_1,   1'R^-1 Y = 1'x_y + a'z_y,   mu = their ratio,
//   Q = (Y - 1 mu)'(x_y - mu x_1) + (b - mu a)'(z_y - mu z_1),
//   Y'R^-1 Y = Y'x_y + b'z_y,
// a = L^-1 1, b = L^-1 Y (columns 8, 9).  A further step first applies the
// backward substitution to z and adds it to x.
//
// Stopping rule.  The factor's pivots carry an absolute error of about
// u (1 + delta) each, u = 2^-8s for s slices in the trailing updates (2^-40
// at the default 5: a row of L has norm^2 R_ii = 1 + delta and the split
// products are exact to about u of it), so log|R| = sum log L_ii^2 is
// uncertain by about e_ld = u (1 + delta) sum_i 1 / L_ii^2.  Step k
// changes n log Q by dq_k; with the contraction rho of the iteration (1/16
// assumed after the first step, then dq_k / dq_{k-1}) the error of n log Q
// left is about dq_k rho / (1 - rho).  Once that is below e_ld, further steps
// cannot make -2logL more accurate, and the candidate stops.
// 2^-8s, the accuracy unit of a factor with s slices in its trailing updates
__device__ __forceinline__ double split_unit(int s) {
    return __longlong_as_double((long long)(1023 - 8 * s) << 52);
}

__global__ void __launch_bounds__(kSolveThreads) k_refine_check(MixedBatch b, int step) {
    __shared__ dfl red[kSolveThreads / 32];
    const int t = blockIdx.x;
    InstState* st = b.st + t;
    if (st->status != GP_OK || st->refine_done) return;
    const int n = b.n;
    const float2* x1 = zcol(b, t, 0);
    const float2* xy = zcol(b, t, 1);
    const float2* z1 = zcol(b, t, 2);
    const float2* zy = zcol(b, t, 3);
    const float2* av = zcol(b, t, 8);
    const float2* bv = zcol(b, t, 9);
    const bool corr = step > 0;
    dfl sa = {0.f, 0.f}, sb = {0.f, 0.f}, sc = {0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += kSolveThreads) {
        const dfl c = df_load(xy + i);
        sa = df_add(sa, df_load(x1 + i));
        sb = df_add(sb, c);
        sc = df_fma(df_from_double(b.y[i]), c, sc);
        if (corr) {
            const dfl ai = df_load(av + i), zyi = df_load(zy + i);
            sa = df_fma(ai, df_load(z1 + i), sa);
            sb = df_fma(ai, zyi, sb);
            sc = df_fma(df_load(bv + i), zyi, sc);
        }
    }
    const double A = df_to_double(block_sum_df(sa, red));
    const double B = df_to_double(block_sum_df(sb, red));
    const double C = df_to_double(block_sum_df(sc, red));
    const double m = B / A;
    const dfl md = df_from_double(m);
    dfl sq = {0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += kSolveThreads) {
        const dfl e = df_sub(df_from_double(b.y[i]), md);
        sq = df_fma(e, df_fms(md, df_load(x1 + i), df_load(xy + i)), sq);
        if (corr) {
            const dfl u = df_fms(md, df_load(av + i), df_load(bv + i));
            sq = df_fma(u, df_fms(md, df_load(z1 + i), df_load(zy + i)), sq);
        }
    }
    const double Q = df_to_double(block_sum_df(sq, red));
    if (threadIdx.x == 0) {
        const double Qprev = st->Q;
        st->aa = A;
        st->ab = B;
        st->bb = C;
        st->mu = m;
        st->Q = Q;
        if (!(Q > 0.0)) {
            st->refine_done = 1;            // degenerate: the finalisation reports it
        } else if (corr) {
            const double dq = n * fabs(log(Q) - log(Qprev));
            double rho = 0.0625;
            if (step > 1 && st->dq_prev > 0.0) rho = fmin(0.5, fmax(dq / st->dq_prev, 1.52587890625e-05));
            const double rest = dq * rho / (1.0 - rho);
            const double e_ld = split_unit(b.s) * (1.0 + b.delta) * st->piv_inv;
            st->dq_prev = dq;
            if (rest <= e_ld) st->refine_done = 1;
        }
    }
}

// -2logL = log|R| + n log Q from the sums of the last refinement check; Q is
// taken as zero when Q <= 16 n eps^2 Y'R^-1 Y with eps = 2^-8s, the accuracy
// unit of the split factorisation (2^-40 at 5 slices).
__global__ void k_df_finalize(MixedBatch b, double* nll, double* mu, double* sigma2, double* logdet,
                              int* status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.count) return;
    const InstState st = b.st[t];
    const int n = b.n;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    if (st.status != GP_OK) {
        nll[t] = (st.status == GP_ENOTPD) ? inf : nan;
        mu[t] = nan;
        sigma2[t] = nan;
        if (logdet) logdet[t] = nan;
        status[t] = st.status;
        return;
    }
    const double eps = split_unit(b.s);
    const double Q = st.Q;
    const bool degenerate = !(Q > 16.0 * n * eps * eps * fabs(st.bb));
    nll[t] = degenerate ? -inf : st.logdet + n * log(Q);
    mu[t] = st.mu;
    sigma2[t] = Q / n;
    if (logdet) logdet[t] = st.logdet;
    status[t] = degenerate ? GP_EDEGENERATE : GP_OK;
}

// The kriging weights of one split-precision candidate (v: its one-candidate
// view, the last correction already applied to x): [a | w] as the
// double-float pairs the kriging kernel reads, a = L^-1 1 (column 8) and
// w = x_y - mu x_1 = R^-1 (Y - 1 mu), and the fit's scalars [-2logL, mu,
// sigma2, log|R|, Q, 1'R^-1 1].
__global__ void k_split_model(MixedBatch v, float2* Zm, double* scalars, const double* nll, const int* status,
                              int* status_out) {
    const InstState st = v.st[0];
    const int npad = v.nt * GP_NB;
    const float2* x1 = zcol(v, 0, 0);
    const float2* xy = zcol(v, 0, 1);
    const float2* av = zcol(v, 0, 8);
    const dfl md = df_from_double(st.mu);
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        Zm[i] = av[i];
        df_store(Zm + npad + i, df_fms(md, df_load(x1 + i), df_load(xy + i)));
    }
    if (threadIdx.x == 0) {
        scalars[0] = *nll;
        scalars[1] = st.mu;
        scalars[2] = st.Q / v.n;
        scalars[3] = st.logdet;
        scalars[4] = st.Q;
        scalars[5] = st.aa;
        *status_out = *status;
    }
}

// Convert the double-float factor and solve vectors of one fitted instance
// into the double layout that the kriging kernel reads: L (tiles), a = L^-1 1
// is not needed by the mixed fit, so column 0 of Zd gets x_1 = R^-1 1 and
// column 1 w; the kriging kernel's a'v term is formed from R^-1 1 instead.
__global__ void k_df_to_double(const float2* src, double* dst, size_t count) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const float2 v = src[i];
        dst[i] = (double)v.x + (double)v.y;
    }
}

}  // namespace

cudaError_t launch_diag_mixed(const MixedBatch& b, int J, cudaStream_t s) {
    const size_t smem = (size_t)kPacked * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_diag_mixed, smem, attr);
    if (e != cudaSuccess) return e;
    k_diag_mixed<<<b.count, kDiagThreads, smem, s>>>(b, J);
    return cudaGetLastError();
}

cudaError_t launch_split_panel(const MixedBatch& b, int J, int ns, int gemv, cudaStream_t s) {
    const int m = b.nt - J - 1;
    if (m <= 0) return cudaSuccess;
    k_split_panel<<<dim3(2 * m, b.count), kSplitThreads, 0, s>>>(b, J, ns, gemv);
    return cudaGetLastError();
}

cudaError_t launch_split_fused(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 2;
    if (m <= 0) return cudaSuccess;
    k_split_fused<<<dim3(4 * m, b.count), kSplitThreads, 0, s>>>(b, J);
    return cudaGetLastError();
}

cudaError_t launch_rhs_init(const MixedBatch& b, cudaStream_t s) {
    const int npad = b.nt * GP_NB;
    k_rhs_init<<<dim3((npad + 255) / 256, b.count), 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_df_forward(const MixedBatch& b, int c0, int init, cudaStream_t s) {
    if (init) {
        if (c0 != 0) return cudaErrorInvalidValue;
        cudaError_t e = launch_rhs_init(b, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(b.SC, 0, (size_t)b.count * b.sc_stride * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_fwd_diag<<<b.count, kSubThreads, 0, s>>>(b, c0, 0);
    for (int J = 0; J + 1 < b.nt; ++J)
        k_fwd_tiles<<<dim3(2 * (b.nt - 1 - J), b.count), kSubThreads, 0, s>>>(b, c0, J);
    return cudaGetLastError();
}

cudaError_t launch_df_backward(const MixedBatch& b, int c0, int add_to, cudaStream_t s) {
    const size_t smem = (size_t)GP_NB * kBwdTs * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_bwd_tiles, smem, attr);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.SC, 0, (size_t)b.count * b.sc_stride * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_bwd_diag<<<b.count, kSubThreads, 0, s>>>(b, c0, b.nt - 1, add_to);
    for (int K = b.nt - 1; K > 0; --K)
        k_bwd_tiles<<<dim3(2 * K, b.count), kSubThreads, smem, s>>>(b, c0, K, add_to);
    return cudaGetLastError();
}

cudaError_t launch_df_residual(const MixedBatch& b, cudaStream_t s) {
    const size_t smem = (size_t)kResCols * kTs * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_resid_tiles, smem, attr);
    if (e != cudaSuccess) return e;
    k_resid_tiles<<<dim3(2 * (unsigned)packed_tiles(b.nt), b.count), kResThreads, smem, s>>>(b);
    k_resid_reduce<<<dim3(b.nt, b.count), kResThreads, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_df_finalize(const MixedBatch& b, double* nll, double* mu, double* sigma2, double* logdet,
                               int* status, cudaStream_t s) {
    k_df_finalize<<<(b.count + 127) / 128, 128, 0, s>>>(b, nll, mu, sigma2, logdet, status);
    return cudaGetLastError();
}

cudaError_t launch_split_model(const MixedBatch& v, float2* Zm, double* scalars, const double* nll,
                               const int* status, int* status_out, cudaStream_t s) {
    k_split_model<<<1, 512, 0, s>>>(v, Zm, scalars, nll, status, status_out);
    return cudaGetLastError();
}

cudaError_t launch_keep_forward(const MixedBatch& b, cudaStream_t s) {
    const int npad = b.nt * GP_NB;
    k_keep_forward<<<dim3((2 * npad + 255) / 256, b.count), 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_refine_check(const MixedBatch& b, int step, cudaStream_t s) {
    k_refine_check<<<b.count, kSolveThreads, 0, s>>>(b, step);
    return cudaGetLastError();
}

cudaError_t launch_df_to_double(const float2* src, double* dst, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_df_to_double<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

}  // namespace gp
