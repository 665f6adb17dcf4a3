// k_mixed.cu -- the split-precision (GP_MIXED) factorisation and solves.
//
// Blocked right-looking Cholesky of R(theta) + delta I (Section 3 of the
// paper factors R by Cholesky for the determinant and the solves) with the
// off-diagonal work on the tensor cores:
//
//   diag   L_JJ = chol(A_JJ), W_J = L_JJ^-1        IEEE double (one CTA)
//   panel  L_IJ = A_IJ W_J^T            I > J      split GEMM, tcgen05
//   update A_IK -= L_IJ L_KJ^T      J < K <= I     split GEMM, tcgen05
//
// Split GEMM (after Ozaki, Ogita, Oishi & Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication",
// Numer. Algorithms 59, 2012): each row i of an operand is scaled by 2^(7-E_i)
// (|row| < 2^E_i) and cut into s slices q_a 2^(-8a) with integers |q_a| <= 128,
//     row = 2^(E_i - 7) sum_a q_a 2^(-8a),
// which bf16 holds exactly.  A product of slices summed over the K = 128
// panel columns stays below 2^22 in magnitude, so the tensor core's fp32
// accumulation of the groups a+b = 0 and a+b = 1 is exact; the groups
// a+b >= 2 (weight <= 2^-16) share a third accumulator whose rounding is
// below 2^-40 of the result.  Products with a+b >= s are dropped.  The three
// partial sums are recombined and applied to the working matrix in
// double-float (df.cuh).
//
// Operands reach shared memory by bulk asynchronous copies (cp.async.bulk)
// of pre-swizzled "images": the slicing kernels write each 128-row x 32-col
// bf16 chunk in the 64-byte-swizzled K-major layout the MMA descriptors
// expect, so a chunk is one contiguous 8 KB copy.  Accumulators live in
// tensor memory (3 x 128 of the 512 columns).
//
// Solves: forward and backward substitution with the double-float factor,
// two right-hand sides [1 Y], then iterative refinement against the
// double-float copy of R (residuals r = b - R x).
#include <cuda_bf16.h>
#include <stdint.h>

#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kChunkElems = GP_NB * 32;       // bf16 elements in one 128 x 32 image chunk
constexpr uint32_t kChunkBytes = kChunkElems * 2;
constexpr int kChunks = GP_NB / 32;           // 4 chunks per 128-wide panel
constexpr int kEpiWarps = 8;                  // epilogue warps: kEpiWarps / 4 per tensor-memory lane quarter
                                               // (16 measured 2% slower on the update)
constexpr int kEpiParts = kEpiWarps / 4;       // column parts of a tile
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;   // warp 0 copies, warp 1 MMA, then the epilogue
constexpr int kEpiThreads = 32 * kEpiWarps;
// Early-release kernels (k_split_gemm<..., true>): warpgroup 0 holds the copy
// and MMA warps (and two idle ones) and gives registers up to the
// kEpiWarpsER epilogue warps, which keep a whole column part of a tile's
// combined result in registers.  The split must fit the launch's registers:
// 128 * kRegsLow + 32 * kEpiWarpsER * kRegsHigh <= kGemmThreadsER * (registers
// at launch, 96 for 640 threads).
constexpr int kEpiWarpsER = 16;
constexpr int kEpiPartsER = kEpiWarpsER / 4;
constexpr int kGemmThreadsER = 128 + 32 * kEpiWarpsER;
constexpr int kEpiThreadsER = 32 * kEpiWarpsER;
constexpr int kRegsLow = 32;
constexpr int kRegsHigh = 112;
static_assert(128 * kRegsLow + 32 * kEpiWarpsER * kRegsHigh <= kGemmThreadsER * (65536 / kGemmThreadsER / 8 * 8),
              "register split exceeds the launch's registers");
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // bounded waits: 2 s

// ---------------------------------------------------------------- PTX ------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity, giving up after `limit_ns`, or
// as soon as *abort is set (another role of the CTA gave up).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, const volatile int* abort = nullptr,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try(b, parity)) return true;
        if (abort && *abort) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: start, leading/stride byte offsets, the
// fixed version bit, swizzle mode (4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t mode) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(mode & 7) << 61;
    return d;
}

// Instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Arrive on the barrier at this CTA-relative offset in every CTA of `mask`
// once this thread's earlier MMAs have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(smem_u32(bar)), "h"(mask)
                 : "memory");
}

// Bulk copy into the same CTA-relative shared-memory offset of every CTA in
// `mask`, each copy completing its bytes on that CTA's barrier at `bar`'s offset.
__device__ __forceinline__ void bulk_g2s_mc(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                            uint16_t mask) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster (memory ordered across it).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8-byte asynchronous global -> shared copies (every one of a thread's
// copies in flight at once), then a wait for all of them
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void regs_dec() { asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N)); }
template <int N>
__device__ __forceinline__ void regs_inc() { asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N)); }

// ----------------------------------------------------------- layouts -------

__device__ __forceinline__ float2* df_tile(const MixedBatch& b, float2* base, int t, int I, int J) {
    return base + (size_t)t * b.inst_stride + (size_t)tile_index(I, J, b.nt) * GP_TILE_ELEMS;
}

// slices of row-block I: [slice][chunk][128 x 32 image]
__device__ __forceinline__ __nv_bfloat16* ps_block(const MixedBatch& b, int t, int I) {
    return b.PS + (size_t)t * b.ps_stride + (size_t)I * b.sp * kChunks * kChunkElems;
}
__device__ __forceinline__ int* pe_block(const MixedBatch& b, int t, int I) {
    return b.PE + (size_t)t * b.pe_stride + (size_t)I * GP_NB;
}

// slices of row block I over two panels (256 columns): [slice][8 chunks][128 x 32]
__device__ __forceinline__ __nv_bfloat16* pf_block(const MixedBatch& b, int t, int I) {
    return b.PF + (size_t)t * b.pf_stride + (size_t)I * b.s * 2 * kChunks * kChunkElems;
}
__device__ __forceinline__ int* fe_block(const MixedBatch& b, int t, int I) {
    return b.FE + (size_t)t * b.fe_stride + (size_t)I * GP_NB;
}

// byte offset of the 16-byte piece holding columns k0..k0+7 (k0 % 8 == 0)
// of row r inside a 128 x 32 chunk with 64-byte swizzle
__device__ __forceinline__ uint32_t image_piece(int r, int k0) {
    const uint32_t piece = (uint32_t)((k0 & 31) >> 3);
    const uint32_t sw = piece ^ (uint32_t)((r & 7) >> 1);
    return (uint32_t)(r >> 3) * 512u + (uint32_t)(r & 7) * 64u + sw * 16u;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Cut a double-float x (already scaled so |x| <= 2^7) into s slices: slice a
// is the integer q_a (|q_a| <= 128) times 2^(-8a), so x = sum_a slice_a and
// every product of slices carries its own weight 2^(-8(a+b)) into the
// tensor-core accumulators.
__device__ __forceinline__ void cut_slices(float xh, float xl, int s, float* m) {
    float w = 1.f;
#pragma unroll
    for (int a = 0; a < GP_MAX_SLICES; ++a) {
        if (a < s) {
            const float q = rintf(xh);
            m[a] = __fmul_rn(q, w);
            w = __fmul_rn(w, 0.00390625f);
            const float dh = __fsub_rn(xh, q);   // exact
            two_sum(dh, xl, xh, xl);
            xh = __fmul_rn(xh, 256.f);
            xl = __fmul_rn(xl, 256.f);
        } else {
            m[a] = 0.f;
        }
    }
}

// ----------------------------------------------------------- kernels -------

__device__ __forceinline__ int exponent_of(float mx) {
    // mx = f 2^E with f in [0.5, 1); 0 for mx == 0
    if (mx == 0.f) return 0;
    const int bits = __float_as_int(mx);
    const int be = (bits >> 23) & 0xff;
    if (be != 0) return be - 126;
    int E;
    frexpf(mx, &E);
    return E;
}

// Diagonal block of column J in double-float on the FP32 pipes (an FP64
// instruction costs about 64 FP32 ones here): L_JJ = chol(A_JJ), log-det,
// the reciprocal diagonal, and W = L_JJ^-1 with the slices of W's rows.
// The block lives in shared memory as a packed lower triangle (row-major,
// P[r(r+1)/2 + c]), 66 KB, so that three CTAs share an SM.
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
// the next pivot: 1 / sqrt by a float seed and three Newton steps in double.
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
    // pivot c: 1 / sqrt(a) from a float seed (about 22 correct bits) and two
    // Newton steps in double-float, y <- y + y (1 - a y^2) / 2 (44, then
    // about 48 bits), L_cc = a y; all on the FP32 pipes, since this chain is
    // the sweep's critical path.  Pivots outside [2^-100, 2^100] (the float
    // seed's comfortable range) take the double route.
    auto take_pivot = [&](int c, dfl a) {
        dfl y, l;
        if (!(a.hi > 0.f) || !isfinite(a.hi)) {
            failed = c;
            y = dfl{1.f, 0.f};
            l = y;
        } else if (a.hi > 7.9e-31f && a.hi < 1.26e30f) {
            const float y0 = rsqrtf(a.hi);
            y = dfl{y0, 0.f};
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const dfl e = df_sub(dfl{1.f, 0.f}, df_mul(df_mul(a, y), y));
                y = df_fma(df_mul(dfl{0.5f, 0.f}, y), e, y);
            }
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
            }
        }
        __syncthreads();
        if (c + 1 == GP_NB) break;
        // phase 2: rows i > c, X_ip += L_ic V_p (p <= i), a warp per row; warp
        // 0 takes only row c + 1 and its pivot, the others deal the rest
        dfl vl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) vl[j] = V[lane + 32 * j];
        const int i0 = (warp == 0) ? c + 1 : c + 1 + warp;
        const int di = (warp == 0) ? GP_NB : kWarps - 1;
        for (int i = i0; i < GP_NB; i += di) {
            const dfl m = df_neg(V[i]);    // L_ic
            dfl* row = P + prow(i);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = lane + 32 * j;
                if (p <= i) {
                    const dfl x0 = (p == c) ? dfl{0.f, 0.f} : row[p];
                    const dfl x = df_fma(m, vl[j], x0);
                    if (p == c + 1 && i == c + 1)
                        take_pivot(c + 1, x);
                    else
                        row[p] = x;
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
    if (threadIdx.x < GP_NB) {
        double v = log(df_to_double(lcc[threadIdx.x]));
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) lsum[warp] = v;
        float2* rinv = b.Z + (size_t)t * b.z_stride + (size_t)4 * b.nt * GP_NB + J * GP_NB;
        df_store(rinv + threadIdx.x, dinv[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ld = 0.0;
        for (int w = 0; w < GP_NB / 32; ++w) ld += lsum[w];
        b.st[t].logdet += 2.0 * ld;
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
// k_split_fused: 8 columns of each of two panels per thread, a quarter tile
constexpr int kFusedParts = 16;
constexpr int kFusedRows = kSplitThreads / kFusedParts;
constexpr int kFusedCols = GP_NB / kFusedParts;

// 2^(7 - E) as two exact float factors (7 - E may leave the float range)
__device__ __forceinline__ void slice_scale(int E, float& sa, float& sb) {
    const int e2 = 7 - E;
    const int ea = e2 > 127 ? 127 : (e2 < -126 ? -126 : e2);
    const int eb = e2 - ea;
    sa = __int_as_float((ea + 127) << 23);
    sb = (eb == 0) ? 1.f : __int_as_float(((eb > 127 ? 127 : (eb < -126 ? -126 : eb)) + 127) << 23);
}

// Slices of one thread's NC values of row r (columns k0 .. k0 + NC - 1 of
// image chunk `chunk0`, k0 = 0, 8, 16 or 24; slice a at chunk0 + a *
// slice_bytes): NC / 8 pieces of 8.
template <int NC>
__device__ __forceinline__ void slice_pieces(const float2 (&v)[NC], float sa, float sb, int r, int k0,
                                             int ns, uint8_t* chunk0, size_t slice_bytes) {
#pragma unroll
    for (int h = 0; h < NC / 8; ++h) {
        float xh[8], xl[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            xh[e] = __fmul_rn(__fmul_rn(v[8 * h + e].x, sa), sb);
            xl[e] = __fmul_rn(__fmul_rn(v[8 * h + e].y, sa), sb);
        }
        const uint32_t off = image_piece(r, k0 + 8 * h);
        float w = 1.f;
#pragma unroll
        for (int a = 0; a < GP_MAX_SLICES; ++a) {
            if (a >= ns) break;
            float m[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float qv = rintf(xh[e]);
                m[e] = __fmul_rn(qv, w);
                two_sum(__fsub_rn(xh[e], qv), xl[e], xh[e], xl[e]);
                xh[e] = __fmul_rn(xh[e], 256.f);
                xl[e] = __fmul_rn(xl[e], 256.f);
            }
            w = __fmul_rn(w, 0.00390625f);
            uint4 pk;
            pk.x = pack_bf16x2(m[0], m[1]);
            pk.y = pack_bf16x2(m[2], m[3]);
            pk.z = pack_bf16x2(m[4], m[5]);
            pk.w = pack_bf16x2(m[6], m[7]);
            *reinterpret_cast<uint4*>(chunk0 + (size_t)a * slice_bytes + off) = pk;
        }
    }
}

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
// quarter tile (32 rows); thread (r, part) owns the same 16-byte piece (8
// columns) of each panel and keeps both panels' values in registers for the
// row maximum and the slicing.
__global__ void __launch_bounds__(kSplitThreads) k_split_fused(MixedBatch b, int J) {
    __shared__ float pmax[kFusedParts][kFusedRows];
    __shared__ dfl xs[2][GP_NB];
    __shared__ dfl red[kFusedParts][2][kFusedRows];
    const int t = blockIdx.y;
    if (b.st[t].status != GP_OK) return;
    const int I = J + 2 + blockIdx.x / 4;
    const int rl = threadIdx.x % kFusedRows, part = threadIdx.x / kFusedRows;
    const int q = part >> 2, c0 = kFusedCols * part;
    const int r = (blockIdx.x & 3) * kFusedRows + rl;
    if (b.fwd && threadIdx.x < 2 * GP_NB) {
        // x_{J+1}: the panel J term was applied by k_split_panel
        const int k = threadIdx.x >> 7, c = threadIdx.x & 127;
        xs[k][c] = df_load(b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB + (size_t)(J + 1) * GP_NB + c);
    }
    const float2* src0 = df_tile(b, b.A, t, I, J);
    const float2* src1 = df_tile(b, b.A, t, I, J + 1);
    // both panels' values stay in registers: each tile is read once
    float2 v0[kFusedCols], v1[kFusedCols];
#pragma unroll
    for (int j = 0; j < kFusedCols; ++j) {
        v0[j] = src0[(size_t)(c0 + j) * GP_NB + r];
        v1[j] = src1[(size_t)(c0 + j) * GP_NB + r];
    }
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < kFusedCols; ++j) mx = fmaxf(mx, fmaxf(fabsf(v0[j].x), fabsf(v1[j].x)));
    pmax[part][rl] = mx;
    __syncthreads();
    if (b.fwd) fwd_partials(v1, xs, c0, part, rl, red);
#pragma unroll
    for (int k = 0; k < kFusedParts; ++k) mx = fmaxf(mx, pmax[k][rl]);
    const int E = exponent_of(mx);
    if (part == 0) fe_block(b, t, I)[r] = E;
    float sa, sb;
    slice_scale(E, sa, sb);
    const size_t slice_bytes = (size_t)2 * kChunks * kChunkBytes;
    uint8_t* base = reinterpret_cast<uint8_t*>(pf_block(b, t, I));
    slice_pieces(v0, sa, sb, r, c0 & 31, b.s, base + (size_t)q * kChunkElems * 2, slice_bytes);
    slice_pieces(v1, sa, sb, r, c0 & 31, b.s, base + (size_t)(4 + q) * kChunkElems * 2, slice_bytes);
    if (b.fwd) {
        __syncthreads();
        fwd_apply<kFusedParts>(b, t, I, r, part, rl, red);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// The MMAs of one stage: every slice product (a, bb), a + bb < NS, over the
// stage's two K = 16 steps, into accumulator group min(a + bb, NG - 1).  The
// loops unroll for a compile-time slice count, so each MMA costs its issue
// and two 64-bit adds to descriptors built once per stage (their address
// field, bits 0-13, holds the byte address / 16 and does not overflow inside
// shared memory).  In the first stage of a tile (FIRST) the first product of
// each group -- (0, g), K step 0, in this order -- overwrites the group.
template <int NS, int NG, int NT, uint32_t kBBytes, bool FIRST>
__device__ __forceinline__ void issue_stage(uint32_t tacc, uint64_t ad0, uint64_t bd0, uint32_t idesc) {
#pragma unroll
    for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int bb = 0; a + bb < NS; ++bb) {
            constexpr int kLast = NG - 1;
            const int gr = (a + bb < kLast) ? (a + bb) : kLast;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint64_t ad = ad0 + (uint64_t)((a * kChunkBytes + kk * 32) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((bb * kBBytes + kk * 32) >> 4);
                const bool overwrite = FIRST && a == 0 && kk == 0 && bb <= kLast;
                mma_bf16(tacc + gr * NT, ad, bd, idesc, overwrite ? 0u : 1u);
            }
        }
    }
}

// issue_stage for the runtime slice count (2 .. 7)
template <int NG, int NT, uint32_t kBBytes>
__device__ __forceinline__ void issue_stage_ns(int ns, bool first, uint32_t tacc, uint64_t ad0, uint64_t bd0,
                                               uint32_t idesc) {
#define GP_ISSUE(N)                                                                     \
    if (first) issue_stage<N, NG, NT, kBBytes, true>(tacc, ad0, bd0, idesc);             \
    else       issue_stage<N, NG, NT, kBBytes, false>(tacc, ad0, bd0, idesc);            \
    return
    switch (ns) {
        case 2: GP_ISSUE(2);
        case 3: GP_ISSUE(3);
        case 4: GP_ISSUE(4);
        case 5: GP_ISSUE(5);
        case 6: GP_ISSUE(6);
        default: GP_ISSUE(7);
    }
#undef GP_ISSUE
}

// Split GEMM over 128 x NT output tiles with NG accumulator groups (group g
// gathers the products with a + b = g, the last one all a + b >= g).
// MODE 0 (panel):  A_IJ(:, cols)  =  PS_I . WS(cols)^T   NT = 64, ps slices,
//                  every group exact: the result must stay accurate relative
//                  to |A| |W|, which exceeds |L_IJ| when L_JJ is ill-conditioned.
// MODE 1 (update): A_IK -= PS_I . PS_K^T                  NT = 128, s slices,
//                  groups 0..NG-2 exact, the last rounded (rows of L have
//                  norm <= 1, so nothing amplifies it).
//
// Persistent: one CTA per SM walks the work items w = blockIdx.x + k gridDim.x
// (instance-major).  Warp 0 streams K-chunk stages through a two-slot ring
// that runs on across tiles, so the next tile's operands land while the
// current tile's epilogue runs; warp 1 issues the MMAs once the epilogue has
// drained the accumulators of the previous tile (or, when two accumulator
// sets fit, of the tile before it); the kEpiWarps epilogue warps read tensor
// memory and apply the result (kEpiWarps / 4 warps per tensor-memory lane
// quarter, each taking one column part, with the loads of a column block
// issued together).  Every wait is bounded; a timeout marks the instance
// GP_ETIMEOUT and stops the CTA after its copies and MMAs have landed.
//
// ER (early release; MODE 1, NT = 128 only): the epilogue first reads and
// combines every accumulator group of its columns into registers, releases
// tensor memory to the MMA warp, and only then reads, updates and writes C,
// so that C's round trip overlaps the next tile's MMAs.  Warps 2, 3 idle;
// the epilogue warps are 4 .. 3 + kEpiWarpsER and hold kRegsHigh registers each.
template <int MODE, int NT, int NG, bool ER = false>
__global__ void __launch_bounds__(ER ? kGemmThreadsER : kGemmThreads, 1)
    k_split_gemm(MixedBatch b, int J, int per_inst, int kind) {
    static_assert(NG * NT <= 512, "accumulators exceed tensor memory");
    static_assert(!ER || (MODE == 1 && NT == 128 && NG == 4) || (MODE == 0 && NT == 64),
                  "early release is built for the 128-column update and the panel solve");
    constexpr int kEpiBase = ER ? 4 : 2;          // first epilogue warp
    // two accumulator sets when they fit (64-column update tiles): the MMAs of
    // tile i + 1 then run while the epilogue drains tile i
    constexpr int NBUF = (2 * NG * NT <= 512) ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(8) uint64_t tfull_bar[NBUF];
    __shared__ __align__(8) uint64_t tempty_bar[NBUF];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ __align__(8) uint64_t never_bar;   // never signalled: the timeout test waits on it
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    // kind (MODE 1): 0 trailing tiles from J + 1 (K = 128), 1 the single
    // column J + 1 (look-ahead, K = 128), 2 trailing tiles from J + 2 with
    // the two panels J, J + 1 fused (K = 256)
    const int ns = (MODE == 0) ? b.ps : b.s;
    const bool fused = (MODE == 1 && kind == 2);
    const int nch = fused ? 2 * kChunks : kChunks;
    constexpr uint32_t kBBytes = kChunkBytes / (GP_NB / NT);      // B rows col0..col0+NT of a chunk
    const uint32_t a_bytes = (uint32_t)ns * kChunkBytes;
    const uint32_t stage_bytes = a_bytes + (uint32_t)ns * kBBytes;
    constexpr uint32_t idesc = idesc_bf16(NT);
    const int total = per_inst * b.count;

    // work item -> (instance, I, K, first column)
    auto decode = [&](int w, int& t, int& I, int& K, int& col0) {
        t = w / per_inst;
        const int q = w - t * per_inst;
        const int tile = q / (GP_NB / NT);
        col0 = (q % (GP_NB / NT)) * NT;
        if (MODE == 0) {
            I = J + 1 + tile;
            K = J;
        } else if (kind == 1) {
            I = J + 1 + tile;
            K = J + 1;
        } else {
            int ii, kk;
            tri_decode(tile, ii, kk);
            const int base = (kind == 2) ? J + 2 : J + 1;
            I = base + ii;
            K = base + kk;
        }
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], 1);
        mbar_init(&empty_bar[1], 1);
        for (int u = 0; u < NBUF; ++u) {
            mbar_init(&tfull_bar[u], 1);
            mbar_init(&tempty_bar[u], ER ? kEpiThreadsER : kEpiThreads);
        }
        mbar_init(&drain_bar, 1);
        mbar_init(&never_bar, 1);
        abort_flag = 0;
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

    auto epilogue_er = [&]() {
        // early-release epilogue: warp w reads TMEM lane quarter w % 4 and
        // the column part (w - 4) / 4 of the tile (NT / kEpiPartsER columns)
        const int q = warp & 3;
        const int part = (warp - kEpiBase) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
        constexpr int kPartCols = NT / kEpiPartsER;
        constexpr int CB1 = 8;                  // columns per TMEM load (phase 1)
        constexpr int CB2 = (kPartCols < 16) ? kPartCols : 16;   // columns per C block (phase 2)
        static_assert(kPartCols % CB1 == 0 && kPartCols % CB2 == 0, "column part vs block widths");
        const int ng_used = ns < NG ? ns : NG;
        const int cbase = part * kPartCols;
        int i = 0;
        for (int w = blockIdx.x; w < total && !abort_flag; w += gridDim.x) {
            int t, I, K, col0;
            decode(w, t, I, K, col0);
            if (b.st[t].status != GP_OK) continue;
            float2* C = df_tile(b, b.A, t, I, K) + (size_t)col0 * GP_NB;
            if (MODE == 1 && threadIdx.x == 32 * kEpiBase) prefetch_l2(C, (uint32_t)(NT * GP_NB * sizeof(float2)));
            if (!mbar_wait(&tfull_bar[0], i & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            // phase 1: sum of the groups, as in the epilogue below, for all
            // kPartCols columns of this thread's row
            float hv[kPartCols], lv[kPartCols];
#pragma unroll
            for (int cb = 0; cb < kPartCols; cb += CB1) {
                float d[NG][CB1];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    if (g < ng_used) {
                        if (CB1 == 8) tmem_ld8(lane_addr + g * NT + cbase + cb, d[g]);
                        else          tmem_ld16(lane_addr + g * NT + cbase + cb, d[g]);
                    } else {
#pragma unroll
                        for (int j = 0; j < CB1; ++j) d[g][j] = 0.f;
                    }
                }
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < CB1; ++j) {
                    float h, l;
                    two_sum(d[0][j], d[1][j], h, l);
                    if (MODE == 1) {
#pragma unroll
                        for (int g = 2; g < NG - 1; ++g) {
                            float s2, e2;
                            two_sum(h, d[g][j], s2, e2);
                            h = s2;
                            l = __fadd_rn(l, e2);
                        }
                        l = __fadd_rn(l, d[NG - 1][j]);
                        two_sum(h, l, h, l);
                    } else {
#pragma unroll
                        for (int g = 2; g < NG; ++g) {
                            float s2, e2;
                            two_sum(h, d[g][j], s2, e2);
                            l = __fadd_rn(l, e2);
                            fast_two_sum(s2, l, h, l);
                        }
                    }
                    hv[cb + j] = h;
                    lv[cb + j] = l;
                }
            }
            // tensor memory is free for the next tile's MMAs
            tc_fence_before();
            mbar_arrive(&tempty_bar[0]);
            // phase 2: C - 2^e (h + l) (update), or 2^e (h + l) (panel)
            const int eA = ((MODE == 0 || !fused) ? pe_block(b, t, I) : fe_block(b, t, I))[r];
            const int* eBp = ((MODE == 0) ? (b.WE + (size_t)t * b.we_stride)
                                          : (fused ? fe_block(b, t, K) : pe_block(b, t, K))) + col0 + cbase;
#pragma unroll
            for (int cb = 0; cb < kPartCols; cb += CB2) {
                float2 cv[CB2];
                if (MODE == 1) {
#pragma unroll
                    for (int j = 0; j < CB2; ++j) cv[j] = C[(size_t)(cbase + cb + j) * GP_NB + r];
                }
#pragma unroll
                for (int j = 0; j < CB2; ++j) {
                    const int e = eA + __ldg(eBp + cb + j) - 14;
                    const float sc = (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
                    const float h = __fmul_rn(hv[cb + j], sc);
                    const float l = __fmul_rn(lv[cb + j], sc);
                    if (MODE == 0) {
                        float hh, ll;
                        fast_two_sum(h, l, hh, ll);
                        C[(size_t)(cbase + cb + j) * GP_NB + r] = make_float2(hh, ll);
                        continue;
                    }
                    float sh, se;
                    two_sum(cv[j].x, -h, sh, se);
                    se = __fadd_rn(se, __fsub_rn(cv[j].y, l));
                    two_sum(sh, se, sh, se);
                    C[(size_t)(cbase + cb + j) * GP_NB + r] = make_float2(sh, se);
                }
            }
            ++i;
        }
    };

    // setmaxnreg is warpgroup-wide: one instruction per warpgroup, every
    // thread of it executing that same instruction
    if (ER && warp >= kEpiBase) {
        regs_inc<kRegsHigh>();
        epilogue_er();
    } else {
    if (ER) regs_dec<kRegsLow>();               // warpgroup 0: copies, MMAs, two idle warps
    if (warp == 0) {
        if (lane == 0) {
            int g = 0;   // stages issued so far
            for (int w = blockIdx.x; w < total && !abort_flag; w += gridDim.x) {
                int t, I, K, col0;
                decode(w, t, I, K, col0);
                if (b.st[t].status != GP_OK) continue;
                const __nv_bfloat16* gA = fused ? pf_block(b, t, I) : ps_block(b, t, I);
                const __nv_bfloat16* gBb = (MODE == 0) ? (b.WS + (size_t)t * b.ws_stride)
                                                       : (fused ? pf_block(b, t, K) : ps_block(b, t, K));
                const uint8_t* gB = reinterpret_cast<const uint8_t*>(gBb) + (size_t)col0 * 64;   // 64 B per row in a chunk
                for (int kc = 0; kc < nch; ++kc, ++g) {
                    const int st = g & 1;
                    if (g >= 2 && !mbar_wait(&empty_bar[st], ((g >> 1) - 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t* sa = smem + st * stage_bytes;
                    uint8_t* sb = sa + a_bytes;
                    mbar_expect_tx(&full_bar[st], stage_bytes);
                    for (int a = 0; a < ns; ++a)
                        bulk_g2s(sa + a * kChunkBytes, gA + (size_t)(a * nch + kc) * kChunkElems, kChunkBytes,
                                 &full_bar[st]);
                    for (int a = 0; a < ns; ++a)
                        bulk_g2s(sb + a * kBBytes, gB + (size_t)(a * nch + kc) * kChunkBytes, kBBytes,
                                 &full_bar[st]);
                }
            }
            // no copy may still be landing when the CTA retires
            for (int k = (g > 2 ? g - 2 : 0); k < g; ++k) mbar_wait(&full_bar[k & 1], (k >> 1) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, i = 0;   // stages consumed, tiles finished
            for (int w = blockIdx.x; w < total && !abort_flag; w += gridDim.x) {
                int t, I, K, col0;
                decode(w, t, I, K, col0);
                if (b.st[t].status != GP_OK) continue;
                // accumulator set i % NBUF is free once the epilogue has drained
                // tile i - NBUF
                const int buf = i % NBUF;
                if (i >= NBUF && !mbar_wait(&tempty_bar[buf], ((i / NBUF) - 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                // test hook: a wait that nothing ends, limited to 5 ms
                if (b.inject_timeout && J == 0 && blockIdx.x == 0 && i == 0 &&
                    !mbar_wait(&never_bar, 0, &abort_flag, 5000000ull)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                for (int kc = 0; kc < nch; ++kc, ++g) {
                    const int st = g & 1;
                    if (!mbar_wait(&full_bar[st], (g >> 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + st * stage_bytes);
                    const uint32_t sb = sa + a_bytes;
                    const uint64_t ad0 = smem_desc(sa, 16, 512, 4), bd0 = smem_desc(sb, 16, 512, 4);
                    issue_stage_ns<NG, NT, kBBytes>(ns, kc == 0, tbase + buf * NG * NT, ad0, bd0, idesc);
                    mma_commit(&empty_bar[st]);
                }
                if (abort_flag) break;
                mma_commit(&tfull_bar[buf]);
                ++i;
            }
            // every MMA issued has completed before tensor memory is released
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0);
        }
    } else if (!ER) {
        // epilogue: warps 2 .. 1 + kEpiWarps; warp w reads TMEM lane quarter
        // w % 4 and the column part (w - 2) / 4 of the tile
        const int q = warp & 3;
        const int part = (warp - 2) >> 2;       // column part: NT / kEpiParts columns
        const int r = q * 32 + lane;
        const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
        constexpr int kPartCols = NT / kEpiParts;
        constexpr int CB = (NG > 4) ? 8 : 16;               // columns per TMEM load
        static_assert(kPartCols % CB == 0, "column part not a multiple of the TMEM load width");
        // products a + b <= ns - 1 exist, so with ns < NG slices the groups
        // from ns on are never written and read as zero
        const int ng_used = ns < NG ? ns : NG;
        int i = 0;
        for (int w = blockIdx.x; w < total && !abort_flag; w += gridDim.x) {
            int t, I, K, col0;
            decode(w, t, I, K, col0);
            if (b.st[t].status != GP_OK) continue;
            float2* C = df_tile(b, b.A, t, I, K) + (size_t)col0 * GP_NB;
            // the C tile (contiguous) heads for L2 while this tile's MMAs run
            if (MODE == 1 && threadIdx.x == 64) prefetch_l2(C, (uint32_t)(NT * GP_NB * sizeof(float2)));
            const int buf = i % NBUF;
            if (!mbar_wait(&tfull_bar[buf], (i / NBUF) & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int* eAp = fused ? fe_block(b, t, I) : pe_block(b, t, I);
            const int* eBp = ((MODE == 0) ? (b.WE + (size_t)t * b.we_stride)
                                          : (fused ? fe_block(b, t, K) : pe_block(b, t, K))) + col0;
            const int eA = eAp[r];
            for (int c0 = part * kPartCols; c0 < (part + 1) * kPartCols; c0 += CB) {
                float2 cv[CB];
                if (MODE == 1) {
#pragma unroll
                    for (int j = 0; j < CB; ++j) cv[j] = C[(size_t)(c0 + j) * GP_NB + r];
                }
                float d[NG][CB];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    if (g < ng_used) {
                        if (CB == 8) tmem_ld8(lane_addr + buf * NG * NT + g * NT + c0, d[g]);
                        else         tmem_ld16(lane_addr + buf * NG * NT + g * NT + c0, d[g]);
                    } else {
#pragma unroll
                        for (int j = 0; j < CB; ++j) d[g][j] = 0.f;
                    }
                }
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    const int c = c0 + j;
                    // v = sum_g d_g (weights already in the slices).  In the update
                    // the groups 0 .. NG-2 enter exactly and the last (weight
                    // <= 2^-24 of the result) folds into the low word; the panel
                    // keeps every group exact in the double-float sum.
                    float h, l;
                    two_sum(d[0][j], d[1][j], h, l);
                    if (MODE == 1) {
#pragma unroll
                        for (int g = 2; g < NG - 1; ++g) {
                            float s2, e2;
                            two_sum(h, d[g][j], s2, e2);
                            h = s2;
                            l = __fadd_rn(l, e2);
                        }
                        if (NG > 2) l = __fadd_rn(l, d[NG - 1][j]);
                        // h may be tiny under cancellation: normalise without
                        // assuming |h| >= |l|
                        two_sum(h, l, h, l);
                    } else {
#pragma unroll
                        for (int g = 2; g < NG; ++g) {
                            float s2, e2;
                            two_sum(h, d[g][j], s2, e2);
                            l = __fadd_rn(l, e2);
                            fast_two_sum(s2, l, h, l);
                        }
                    }
                    const int e = eA + __ldg(eBp + c) - 14;
                    const float sc = (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
                    h = __fmul_rn(h, sc);
                    l = __fmul_rn(l, sc);
                    float2* p = C + (size_t)c * GP_NB + r;
                    if (MODE == 0) {
                        float hh, ll;
                        fast_two_sum(h, l, hh, ll);
                        *p = make_float2(hh, ll);
                    } else {
                        // C - (h + l) to an absolute error of about 2^-47 (|C| + |h|);
                        // the final normalisation makes no assumption on the
                        // sizes (the diagonal cancels heavily)
                        float sh, se;
                        two_sum(cv[j].x, -h, sh, se);
                        se = __fadd_rn(se, __fsub_rn(cv[j].y, l));
                        two_sum(sh, se, sh, se);
                        *p = make_float2(sh, se);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[buf]);
            ++i;
        }
    }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_flag && threadIdx.x == 0) {
        // every instance this CTA touches is incomplete: later kernels skip
        // them and their outputs read GP_ETIMEOUT
        atomicExch(b.err, GP_ETIMEOUT);
        for (int w = blockIdx.x; w < total; w += gridDim.x) b.st[w / per_inst].status = GP_ETIMEOUT;
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

// Row-pair decode for the fused update run by CTA pairs: the trailing
// triangle's row ii holds tiles kk = 0 .. ii, taken two at a time, so row ii
// has ii / 2 + 1 pairs and rows 0 .. ii - 1 hold h (h + 1) pairs (ii = 2h) or
// h^2 (ii = 2h - 1).  q -> (ii, pair in the row).
__device__ __forceinline__ void pair_decode(int q, int& ii, int& pr) {
    int h = (int)sqrtf((float)q);
    while (h * h > q) --h;
    while ((h + 1) * (h + 1) <= q) ++h;
    if (q >= h * (h + 1)) {
        ii = 2 * h;
        pr = q - h * (h + 1);
    } else {
        ii = 2 * h - 1;
        pr = q - h * h;
    }
}

__host__ __device__ __forceinline__ int pairs_in_triangle(int m) {
    const int h = m / 2;
    return (m % 2 == 0) ? h * (h + 1) : (h + 1) * (h + 1);
}

// The fused (K = 256) trailing update of a panel pair by clusters of two
// CTAs.  The two CTAs of a cluster take the tiles (I, K) and (I, K + 1) of
// one row: they share the A operand (the two-panel slices of row block I),
// so each CTA bulk-copies half of A's slices, multicast into both CTAs'
// shared memory, and its own B; per SM that is three quarters of the
// operand traffic of k_split_gemm, whose trailing updates are bound by it.
// A stage is refilled only when both CTAs' MMAs have read it: every MMA
// commit arrives on both CTAs' empty barriers.  When a row has an odd number
// of tiles, the second CTA of its last pair only supplies its half of A.
// Everything else (MMA groups, exact recombination, bounded waits) is that of
// k_split_gemm<1, 128, 4>.
__global__ void __launch_bounds__(kGemmThreads, 1) k_split_gemm_pair(MixedBatch b, int J, int pairs_per_inst) {
    constexpr int NT = 128, NG = 4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(8) uint64_t tfull_bar;
    __shared__ __align__(8) uint64_t tempty_bar;
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int ns = b.s;
    constexpr int nch = 2 * kChunks;                             // K = 256
    constexpr uint32_t kBBytes = kChunkBytes;                    // NT = 128: whole chunk rows
    const uint32_t a_bytes = (uint32_t)ns * kChunkBytes;
    const uint32_t stage_bytes = a_bytes + (uint32_t)ns * kBBytes;
    constexpr uint32_t idesc = idesc_bf16(NT);
    constexpr uint16_t kPair = 0x3;
    const int rank = (int)cluster_ctarank();
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
    const int total = pairs_per_inst * b.count;

    // pair item -> (instance, I, K, this CTA's tile exists)
    auto decode = [&](int w, int& t, int& I, int& K, bool& valid) {
        t = w / pairs_per_inst;
        int ii, pr;
        pair_decode(w - t * pairs_per_inst, ii, pr);
        const int kk = 2 * pr + rank;
        valid = (kk <= ii);
        I = J + 2 + ii;
        K = J + 2 + (valid ? kk : ii);
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], 2);   // both CTAs' MMAs
        mbar_init(&empty_bar[1], 2);
        mbar_init(&tfull_bar, 1);
        mbar_init(&tempty_bar, kEpiThreads);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    // the partner's barriers exist before any copy or commit targets them
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            for (int w = cid; w < total && !abort_flag; w += ncl) {
                int t, I, K;
                bool valid;
                decode(w, t, I, K, valid);
                if (b.st[t].status != GP_OK) continue;       // the partner skips it too
                const __nv_bfloat16* gA = pf_block(b, t, I);
                const uint8_t* gB = reinterpret_cast<const uint8_t*>(pf_block(b, t, K));
                for (int kc = 0; kc < nch; ++kc, ++g) {
                    const int st = g & 1;
                    if (g >= 2 && !mbar_wait(&empty_bar[st], ((g >> 1) - 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    uint8_t* sa = smem + st * stage_bytes;
                    uint8_t* sb = sa + a_bytes;
                    // this CTA receives all of A (half from each CTA) and its own B
                    mbar_expect_tx(&full_bar[st], a_bytes + (valid ? (uint32_t)ns * kBBytes : 0u));
                    for (int a = rank; a < ns; a += 2)
                        bulk_g2s_mc(sa + a * kChunkBytes, gA + (size_t)(a * nch + kc) * kChunkElems, kChunkBytes,
                                    &full_bar[st], kPair);
                    if (valid)
                        for (int a = 0; a < ns; ++a)
                            bulk_g2s(sb + a * kBBytes, gB + (size_t)(a * nch + kc) * kChunkBytes, kBBytes,
                                     &full_bar[st]);
                }
            }
            // every copy into this CTA (its own and the partner's) has landed,
            // and both CTAs' commits for the last stages have arrived here,
            // before the CTA retires
            for (int k = (g > 2 ? g - 2 : 0); k < g; ++k) mbar_wait(&full_bar[k & 1], (k >> 1) & 1);
            for (int k = (g > 2 ? g - 2 : 0); k < g; ++k) mbar_wait(&empty_bar[k & 1], (k >> 1) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, i = 0;
            for (int w = cid; w < total && !abort_flag; w += ncl) {
                int t, I, K;
                bool valid;
                decode(w, t, I, K, valid);
                if (b.st[t].status != GP_OK) continue;
                if (valid && i >= 1 && !mbar_wait(&tempty_bar, (i - 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                for (int kc = 0; kc < nch; ++kc, ++g) {
                    const int st = g & 1;
                    if (!mbar_wait(&full_bar[st], (g >> 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    if (valid) {
                        const uint32_t sa = smem_u32(smem + st * stage_bytes);
                        const uint32_t sb = sa + a_bytes;
                        const uint64_t ad0 = smem_desc(sa, 16, 512, 4), bd0 = smem_desc(sb, 16, 512, 4);
                        issue_stage_ns<NG, NT, kBBytes>(ns, kc == 0, tbase, ad0, bd0, idesc);
                    }
                    // this stage may be refilled in both CTAs once both have read it
                    mma_commit_mc(&empty_bar[st], kPair);
                }
                if (abort_flag) break;
                if (valid) {
                    mma_commit(&tfull_bar);
                    ++i;
                }
            }
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0);
        }
    } else {
        const int q = warp & 3;
        const int part = (warp - 2) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
        constexpr int kPartCols = NT / kEpiParts;
        constexpr int CB = 16;
        const int ng_used = ns < NG ? ns : NG;
        int i = 0;
        for (int w = cid; w < total && !abort_flag; w += ncl) {
            int t, I, K;
            bool valid;
            decode(w, t, I, K, valid);
            if (b.st[t].status != GP_OK || !valid) continue;
            float2* C = df_tile(b, b.A, t, I, K);
            if (threadIdx.x == 64) prefetch_l2(C, (uint32_t)(NT * GP_NB * sizeof(float2)));
            if (!mbar_wait(&tfull_bar, i & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int eA = fe_block(b, t, I)[r];
            const int* eBp = fe_block(b, t, K);
            for (int c0 = part * kPartCols; c0 < (part + 1) * kPartCols; c0 += CB) {
                float2 cv[CB];
#pragma unroll
                for (int j = 0; j < CB; ++j) cv[j] = C[(size_t)(c0 + j) * GP_NB + r];
                float d[NG][CB];
#pragma unroll
                for (int gq = 0; gq < NG; ++gq) {
                    if (gq < ng_used) {
                        tmem_ld16(lane_addr + gq * NT + c0, d[gq]);
                    } else {
#pragma unroll
                        for (int j = 0; j < CB; ++j) d[gq][j] = 0.f;
                    }
                }
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    const int c = c0 + j;
                    // groups 0 .. 2 exact, the last (weight <= 2^-24) in the low word
                    float h, l;
                    two_sum(d[0][j], d[1][j], h, l);
                    {
                        float s2, e2;
                        two_sum(h, d[2][j], s2, e2);
                        h = s2;
                        l = __fadd_rn(l, e2);
                    }
                    l = __fadd_rn(l, d[3][j]);
                    two_sum(h, l, h, l);
                    const int e = eA + __ldg(eBp + c) - 14;
                    const float sc = (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
                    h = __fmul_rn(h, sc);
                    l = __fmul_rn(l, sc);
                    float sh, se;
                    two_sum(cv[j].x, -h, sh, se);
                    se = __fadd_rn(se, __fsub_rn(cv[j].y, l));
                    two_sum(sh, se, sh, se);
                    C[(size_t)c * GP_NB + r] = make_float2(sh, se);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar);
            ++i;
        }
    }
    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still copy into it or arrive on it
    cluster_sync_all();
    tc_fence_after();
    if (abort_flag && threadIdx.x == 0) {
        atomicExch(b.err, GP_ETIMEOUT);
        for (int w = cid; w < total; w += ncl) b.st[w / pairs_per_inst].status = GP_ETIMEOUT;
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
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
    return b.st[t].status == GP_OK && !b.st[t].hager_done;
}

__device__ __forceinline__ float2* rp_part(const MixedBatch& b, int t, int I, int J) {
    return b.RP + (size_t)t * b.rp_stride + (size_t)tile_index(I, J, b.nt) * kRpTile;
}

// forward, block J: z_J <- W_J (z_J - sum_{K<J} L_JK z_K), W_J = L_JJ^-1
// (column-major WT: thread (k, r) reads row r of W along its columns)
__global__ void __launch_bounds__(kSubThreads) k_fwd_diag(MixedBatch b, int c0, int J) {
    __shared__ dfl rhs[2][GP_NB];
    const int t = blockIdx.x;
    if (!sub_active(b, t)) return;
    const int k = threadIdx.x >> 7, r = threadIdx.x & 127;
    float2* z = zcol(b, t, c0 + k) + (size_t)J * GP_NB;
    dfl v = df_load(z + r);
#pragma unroll 4
    for (int K = 0; K < J; ++K) {
        const float2* pp = rp_part(b, t, J, K) + k * GP_NB + r;
        v = df_sub(v, df_add(df_load(pp), df_load(pp + 2 * GP_NB)));
    }
    rhs[k][r] = v;
    __syncthreads();
    // all 128 columns (W is zero above its diagonal): a fixed trip count
    // lets the loads run ahead of the four accumulation chains
    const float2* W = b.WT + (size_t)t * b.wt_stride + (size_t)J * GP_TILE_ELEMS;
    dfl x[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 16
    for (int c = 0; c < GP_NB; ++c) x[c & 3] = df_fma(df_load(W + (size_t)c * GP_NB + r), rhs[k][c], x[c & 3]);
    df_store(z + r, df_add(df_add(x[0], x[1]), df_add(x[2], x[3])));
}

// forward, tiles (I, J), I > J, half h of the columns: L_IJ(:, h) z_J(h)
__global__ void __launch_bounds__(kSubThreads) k_fwd_tiles(MixedBatch b, int c0, int J) {
    __shared__ dfl xs[2][GP_NB / 2];
    __shared__ dfl part[2][2][GP_NB];
    const int t = blockIdx.y;
    if (!sub_active(b, t)) return;
    const int I = J + 1 + (blockIdx.x >> 1), h = blockIdx.x & 1;
    const int tid = threadIdx.x;
    // W_{J+1} heads for L2 for the next diagonal step
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
}

// backward, block K: z_K <- W_K^T (z_K - sum_{K' > K} L_K'K^T z_K'); W^T
// from the row-major copy WR (thread (k, c) reads column c of W along its
// rows); with add_to >= 0 the result is also added into (add_to, add_to + 1)
__global__ void __launch_bounds__(kSubThreads) k_bwd_diag(MixedBatch b, int c0, int K, int add_to) {
    __shared__ dfl rhs[2][GP_NB];
    const int t = blockIdx.x;
    if (!sub_active(b, t)) return;
    const int nt = b.nt;
    const int k = threadIdx.x >> 7, c = threadIdx.x & 127;
    float2* z = zcol(b, t, c0 + k) + (size_t)K * GP_NB;
    dfl v = df_load(z + c);
#pragma unroll 4
    for (int K2 = K + 1; K2 < nt; ++K2) {
        const float2* pp = rp_part(b, t, K2, K) + k * GP_NB + c;
        v = df_sub(v, df_add(df_load(pp), df_load(pp + 2 * GP_NB)));
    }
    rhs[k][c] = v;
    __syncthreads();
    // all 128 rows (W is zero above its diagonal): a fixed trip count lets
    // the loads run ahead of the four accumulation chains
    const float2* Wr = b.WR + (size_t)t * b.wt_stride + (size_t)K * GP_TILE_ELEMS;
    dfl xa[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 16
    for (int r = 0; r < GP_NB; ++r) xa[r & 3] = df_fma(df_load(Wr + (size_t)r * GP_NB + c), rhs[k][r], xa[r & 3]);
    const dfl x = df_add(df_add(xa[0], xa[1]), df_add(xa[2], xa[3]));
    df_store(z + c, x);
    if (add_to >= 0) {
        float2* acc = zcol(b, t, add_to + k) + (size_t)K * GP_NB + c;
        df_store(acc, df_add(df_load(acc), x));
    }
}

// backward, tiles (K, I), I < K, half h of the rows: L_KI(h, :)^T z_K(h);
// the half tile is staged column by column (64 rows + 1 of padding) so that
// thread c walks column c conflict-free
constexpr int kBwdTs = GP_NB / 2 + 1;
__global__ void __launch_bounds__(kSubThreads) k_bwd_tiles(MixedBatch b, int c0, int K) {
    extern __shared__ dfl T[];                  // GP_NB x kBwdTs
    __shared__ dfl xs[2][GP_NB / 2];
    __shared__ dfl part[2][2][GP_NB];
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
    if (b.st[t].status != GP_OK) return;
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
    if (b.st[t].status != GP_OK) return;
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

// mu_hat = 1'x_y / 1'x_1, w = x_y - mu x_1 = R^-1 (Y - 1 mu), Q = (Y - 1 mu)'w,
// -2logL = log|R| + n log Q; column 1 becomes w (for kriging), column 0 keeps
// x_1 = R^-1 1.  Q is taken as zero when Q <= 16 n eps^2 Y'x_y with
// eps = 2^-40, the accuracy unit of the split factorisation.
__global__ void __launch_bounds__(kSolveThreads) k_df_finalize(MixedBatch b, double* nll, double* mu,
                                                               double* sigma2, double* logdet, int* status) {
    __shared__ dfl red[kSolveThreads / 32];
    const int t = blockIdx.x;
    InstState st = b.st[t];
    const int n = b.n;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    if (st.status != GP_OK) {
        if (threadIdx.x == 0) {
            nll[t] = (st.status == GP_ENOTPD) ? inf : nan;
            mu[t] = nan;
            sigma2[t] = nan;
            if (logdet) logdet[t] = (st.status == GP_ENOTPD) ? nan : nan;
            status[t] = st.status;
        }
        return;
    }
    float2* x1 = zcol(b, t, 0);
    float2* xy = zcol(b, t, 1);
    dfl sa = {0.f, 0.f}, sb = {0.f, 0.f}, sc = {0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += kSolveThreads) {
        const dfl a = df_load(x1 + i), c = df_load(xy + i);
        const dfl yi = df_from_double(b.y[i]);
        sa = df_add(sa, a);
        sb = df_add(sb, c);
        sc = df_fma(yi, c, sc);
    }
    const double A = df_to_double(block_sum_df(sa, red));
    const double B = df_to_double(block_sum_df(sb, red));
    const double C = df_to_double(block_sum_df(sc, red));
    const double m = B / A;
    const dfl md = df_from_double(m);
    dfl sq = {0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += kSolveThreads) {
        const dfl wv = df_fms(md, df_load(x1 + i), df_load(xy + i));
        df_store(xy + i, wv);
        const dfl e = df_sub(df_from_double(b.y[i]), md);
        sq = df_fma(e, wv, sq);
    }
    const double Q = df_to_double(block_sum_df(sq, red));
    if (threadIdx.x == 0) {
        const double eps = 9.094947017729282e-13;   // 2^-40
        const bool degenerate = Q <= 16.0 * n * eps * eps * fabs(C);
        nll[t] = degenerate ? -inf : st.logdet + n * log(Q);
        mu[t] = m;
        sigma2[t] = Q / n;
        if (logdet) logdet[t] = st.logdet;
        status[t] = degenerate ? GP_EDEGENERATE : GP_OK;
        st.aa = A;
        st.ab = B;
        st.bb = C;
        st.mu = m;
        st.Q = Q;
        b.st[t] = st;
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

// SMs of the current device (looked up once per device ordinal)
static int sm_count() {
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < kMaxDevices;
    int n = cached ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        if (cached) cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int MODE, int NT, int NG, bool ER = false>
static cudaError_t launch_gemm(const MixedBatch& b, int J, int per_inst, int ns, cudaStream_t s, int kind = 0) {
    const size_t smem = (size_t)2 * ns * (kChunkBytes + kChunkBytes / (GP_NB / NT)) + 1024;
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_split_gemm<MODE, NT, NG, ER>, smem, attr);
    if (e != cudaSuccess) return e;
    const long long total = (long long)per_inst * b.count;
    const int grid = (int)(total < sm_count() ? total : sm_count());
    k_split_gemm<MODE, NT, NG, ER><<<grid, ER ? kGemmThreadsER : kGemmThreads, smem, s>>>(b, J, per_inst, kind);
    return cudaGetLastError();
}

// The early-release kernels raise their epilogue warps to kRegsHigh
// registers; that only completes if the block was launched with enough
// registers for the whole split, so they run only where the built kernel's
// register count covers it (checked once per device and kernel), else the
// plain kernel runs.
template <int MODE, int NT, int NG>
static bool early_release_fits() {
    static std::atomic<int> ok[kMaxDevices];   // 0 unknown, 1 yes, 2 no
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < kMaxDevices;
    int v = cached ? ok[dev].load(std::memory_order_relaxed) : 0;
    if (v == 0) {
        cudaFuncAttributes fa{};
        v = 2;
        if (cudaFuncGetAttributes(&fa, k_split_gemm<MODE, NT, NG, true>) == cudaSuccess &&
            128 * kRegsLow + 32 * kEpiWarpsER * kRegsHigh <= kGemmThreadsER * fa.numRegs &&
            fa.maxThreadsPerBlock >= kGemmThreadsER)
            v = 1;
        cudaGetLastError();
        if (cached) ok[dev].store(v, std::memory_order_relaxed);
    }
    return v == 1;
}

static cudaError_t launch_update128(const MixedBatch& b, int J, int per_inst, int ns, cudaStream_t s, int kind) {
    if (early_release_fits<1, 128, 4>()) return launch_gemm<1, 128, 4, true>(b, J, per_inst, ns, s, kind);
    return launch_gemm<1, 128, 4>(b, J, per_inst, ns, s, kind);
}

cudaError_t launch_gemm_panel(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 1;
    if (m <= 0) return cudaSuccess;
    if (early_release_fits<0, 64, GP_PANEL_SLICES>())
        return launch_gemm<0, 64, GP_PANEL_SLICES, true>(b, J, 2 * m, b.ps, s);
    return launch_gemm<0, 64, GP_PANEL_SLICES>(b, J, 2 * m, b.ps, s);
}

// Trailing updates with 128-column output tiles, or 64-column ones (twice the
// work items: better load balance for small problems, each output element
// computed by the same products in the same order).
cudaError_t launch_gemm_update_column(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 1;
    if (m <= 0) return cudaSuccess;
    if (b.update_tile == 64) return launch_gemm<1, 64, 4>(b, J, 2 * m, b.s, s, 1);
    return launch_update128(b, J, m, b.s, s, 1);
}

// The fused update by CTA pairs (k_split_gemm_pair): a cluster launch whose
// grid is as many pairs as can be resident at once (looked up per device).
static cudaError_t launch_gemm_pair(const MixedBatch& b, int J, int m, cudaStream_t s) {
    const size_t smem = (size_t)2 * b.s * (2 * kChunkBytes) + 1024;
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_split_gemm_pair, smem, attr);
    if (e != cudaSuccess) return e;
    const int ppi = pairs_in_triangle(m);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static std::atomic<int> clusters[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    int nc = (dev >= 0 && dev < kMaxDevices) ? clusters[dev].load(std::memory_order_relaxed) : 0;
    if (nc == 0) {
        cfg.gridDim = dim3(2 * sm_count());
        e = cudaOccupancyMaxActiveClusters(&nc, k_split_gemm_pair, &cfg);
        if (e != cudaSuccess) return e;
        if (nc < 1) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < kMaxDevices) clusters[dev].store(nc, std::memory_order_relaxed);
    }
    const long long total = (long long)ppi * b.count;
    const int ncl = (int)(total < nc ? total : nc);
    cfg.gridDim = dim3(2 * ncl);
    return cudaLaunchKernelEx(&cfg, k_split_gemm_pair, b, J, ppi);
}

cudaError_t launch_gemm_update_fused(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 2;
    if (m <= 0) return cudaSuccess;
    if (b.update_tile == 64) return launch_gemm<1, 64, 4>(b, J, m * (m + 1), b.s, s, 2);
    if (b.pair_update) return launch_gemm_pair(b, J, m, s);
    return launch_update128(b, J, m * (m + 1) / 2, b.s, s, 2);
}

cudaError_t launch_split_fused(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 2;
    if (m <= 0) return cudaSuccess;
    k_split_fused<<<dim3(4 * m, b.count), kSplitThreads, 0, s>>>(b, J);
    return cudaGetLastError();
}

cudaError_t launch_gemm_update(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 1;
    if (m <= 0) return cudaSuccess;
    const int tiles = m * (m + 1) / 2;
    switch (b.ug) {
        case 7: return launch_gemm<1, 64, 7>(b, J, 2 * tiles, b.s, s);
        case 3: return launch_gemm<1, 128, 3>(b, J, tiles, b.s, s);
        default:
            if (b.update_tile == 64) return launch_gemm<1, 64, 4>(b, J, 2 * tiles, b.s, s);
            return launch_update128(b, J, tiles, b.s, s, 0);
    }
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
    for (int J = 0; J < b.nt; ++J) {
        k_fwd_diag<<<b.count, kSubThreads, 0, s>>>(b, c0, J);
        if (J + 1 < b.nt) k_fwd_tiles<<<dim3(2 * (b.nt - 1 - J), b.count), kSubThreads, 0, s>>>(b, c0, J);
    }
    return cudaGetLastError();
}

cudaError_t launch_df_backward(const MixedBatch& b, int c0, int add_to, cudaStream_t s) {
    const size_t smem = (size_t)GP_NB * kBwdTs * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_bwd_tiles, smem, attr);
    if (e != cudaSuccess) return e;
    for (int K = b.nt - 1; K >= 0; --K) {
        k_bwd_diag<<<b.count, kSubThreads, 0, s>>>(b, c0, K, add_to);
        if (K > 0) k_bwd_tiles<<<dim3(2 * K, b.count), kSubThreads, smem, s>>>(b, c0, K);
    }
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
    k_df_finalize<<<b.count, kSolveThreads, 0, s>>>(b, nll, mu, sigma2, logdet, status);
    return cudaGetLastError();
}

cudaError_t launch_df_to_double(const float2* src, double* dst, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_df_to_double<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

}  // namespace gp
