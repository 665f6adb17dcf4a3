// k_gemm.cu -- the split GEMMs of the split-precision (GP_MIXED) factorisation
// on the tensor cores: the panel solve L_IJ = A_IJ W_J^T and the trailing
// updates A_IK -= L_IJ L_KJ^T (single panels and fused panel pairs),
// each over bf16 slices (mixed_common.cuh) with fp32 accumulation in tensor
// memory and the exact recombination and application in double-float.
// The slicing, the diagonal blocks and the solves are in k_mixed.cu.
#include "mixed_common.cuh"

namespace gp {

namespace {

constexpr int kEpiWarps = 8;                  // epilogue warps of the plain kernels: kEpiWarps / 4 per
                                               // tensor-memory lane quarter
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

// The MMAs of one stage: every slice product (a, bb), a + bb < NS, over the
// stage's two K = 16 steps, into accumulator group min(a + bb, NG - 1).  The
// loops unroll for a compile-time slice count, so each MMA costs its issue
// and two 64-bit adds to descriptors built once per stage (their address
// field, bits 0-13, holds the byte address / 16 and does not overflow inside
// shared memory).  In the first stage of a tile (FIRST) the first product of
// each group -- (0, g), K step 0, in this order -- overwrites the group.
// Only the products of groups GLO .. GHI are issued, each group's in the
// order above: the first stage of a tile can then be issued group by group
// as the epilogue frees the accumulators, every group still accumulating the
// same products in the same order.
template <int NS, int NG, int NT, uint32_t kBBytes, bool FIRST, int GLO = 0, int GHI = NG - 1>
__device__ __forceinline__ void issue_stage(uint32_t tacc, uint64_t ad0, uint64_t bd0, uint32_t idesc) {
#pragma unroll
    for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int bb = 0; a + bb < NS; ++bb) {
            constexpr int kLast = NG - 1;
            const int gr = (a + bb < kLast) ? (a + bb) : kLast;
            if (gr < GLO || gr > GHI) continue;
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
template <int NG, int NT, uint32_t kBBytes, int GLO = 0, int GHI = NG - 1>
__device__ __forceinline__ void issue_stage_ns(int ns, bool first, uint32_t tacc, uint64_t ad0, uint64_t bd0,
                                               uint32_t idesc) {
#define GP_ISSUE(N)                                                                        \
    if (first) issue_stage<N, NG, NT, kBBytes, true, GLO, GHI>(tacc, ad0, bd0, idesc);      \
    else       issue_stage<N, NG, NT, kBBytes, false, GLO, GHI>(tacc, ad0, bd0, idesc);     \
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

// The first stage of a tile in the early-release kernels, group by group: the
// products of groups 0 and 1 once the epilogue has read those two groups of
// the previous tile (release barrier 1), then those of each group G >= 2 once
// it has read group G (barrier G).  False if a wait gave up.
template <int NG, int NT, uint32_t kBBytes, int G = 1>
__device__ __forceinline__ bool issue_first_stage_er(int ns, int i, uint32_t tacc, uint64_t ad0, uint64_t bd0,
                                                     uint32_t idesc, uint64_t* rel, const volatile int* abort) {
    if constexpr (G < NG) {
        if (i >= 1 && !mbar_wait(&rel[G], (i - 1) & 1, abort)) return false;
        tc_fence_after();
        issue_stage_ns<NG, NT, kBBytes, (G == 1 ? 0 : G), G>(ns, true, tacc, ad0, bd0, idesc);
        return issue_first_stage_er<NG, NT, kBBytes, G + 1>(ns, i, tacc, ad0, bd0, idesc, rel, abort);
    }
    return true;
}

// The panel solve's accumulator groups (each exact in fp32) summed into a
// double-float: groups 0 .. 3 through TwoSums, groups 4 .. NG - 1 (weights
// 2^-32 and below of group 0's unit) as one float sum, whose rounding, about
// 2^-56 of that unit, is the slices' own truncation level; one TwoSum
// normalises at the end (h may be small under cancellation).  29 operations
// for 7 groups where a TwoSum and a renormalisation per group took 56, and
// the whole sum precedes the release of tensor memory to the next tile.
template <int NG, int CB>
__device__ __forceinline__ void sum_panel_groups(const float (&d)[NG][CB], int j, float& h, float& l) {
    float e;
    two_sum(d[0][j], d[1][j], h, l);
#pragma unroll
    for (int g = 2; g < NG && g < 4; ++g) {
        two_sum(h, d[g][j], h, e);
        l = __fadd_rn(l, e);
    }
    if (NG > 4) {
        float tail = d[NG - 1][j];
#pragma unroll
        for (int g = NG - 2; g >= 4; --g) tail = __fadd_rn(tail, d[g][j]);
        l = __fadd_rn(l, tail);
    }
    two_sum(h, l, h, l);
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
// ER (early release; the 128-column update and the panel solve, the default
// where the built kernel's registers allow it): the epilogue first reads and
// combines every accumulator group of its columns into registers, releases
// tensor memory to the MMA warp, and only then reads, updates and writes C
// (or stores the panel), so that this overlaps the next tile's MMAs.  In the
// update each group is released as soon as it has been read (groups 0 and 1
// together, then one at a time; the next tile's first stage is issued group
// by group as they come free): 63.8 -> 63.1 ms per step at n = 4000, T = 256.
// The panel solve (7 groups) releases them all at once: group by group it
// took 16.4 -> 17.9 ms.  Warps 2, 3 idle; the epilogue warps are 4 .. 3 +
// kEpiWarpsER and hold kRegsHigh registers each.
template <int MODE, int NT, int NG, bool ER = false>
__global__ void __launch_bounds__(ER ? kGemmThreadsER : kGemmThreads, 1)
    k_split_gemm(MixedBatch b, int J, int per_inst, int kind) {
    static_assert(NG * NT <= 512, "accumulators exceed tensor memory");
    static_assert(!ER || (MODE == 1 && NT == 128 && NG == 4) || (MODE == 0 && NT == 64),
                  "early release is built for the 128-column update and the panel solve");
    constexpr int kEpiBase = ER ? 4 : 2;          // first epilogue warp
    constexpr bool kGroupwise = ER && MODE == 1;   // accumulator groups released one by one
    // two accumulator sets when they fit (64-column update tiles): the MMAs of
    // tile i + 1 then run while the epilogue drains tile i
    constexpr int NBUF = (2 * NG * NT <= 512) ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(8) uint64_t tfull_bar[NBUF];
    __shared__ __align__(8) uint64_t tempty_bar[NBUF];
    __shared__ __align__(8) uint64_t rel_bar[NG];   // early release: group G read (1: groups 0 and 1)
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
        if (kGroupwise)
            for (int g = 1; g < NG; ++g) mbar_init(&rel_bar[g], kEpiThreadsER);
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
            if constexpr (kGroupwise) {
                // group by group (per column the same operations in the same
                // order as one pass over all groups), each released once read
#pragma unroll
                for (int cb = 0; cb < kPartCols; cb += CB1) {
                    float d0[CB1], d1[CB1];
                    tmem_ld8(lane_addr + cbase + cb, d0);
                    if (ng_used > 1) {
                        tmem_ld8(lane_addr + NT + cbase + cb, d1);
                    } else {
#pragma unroll
                        for (int j = 0; j < CB1; ++j) d1[j] = 0.f;
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < CB1; ++j) two_sum(d0[j], d1[j], hv[cb + j], lv[cb + j]);
                }
                tc_fence_before();
                mbar_arrive(&rel_bar[1]);
#pragma unroll
                for (int g = 2; g < NG; ++g) {
                    float dg[kPartCols];
                    if (g < ng_used) {
#pragma unroll
                        for (int cb = 0; cb < kPartCols; cb += CB1) tmem_ld8(lane_addr + g * NT + cbase + cb, dg + cb);
                        tmem_wait_ld();
                    } else {
#pragma unroll
                        for (int j = 0; j < kPartCols; ++j) dg[j] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < kPartCols; ++j) {
                        if (g < NG - 1) {
                            float s2, e2;
                            two_sum(hv[j], dg[j], s2, e2);
                            hv[j] = s2;
                            lv[j] = __fadd_rn(lv[j], e2);
                        } else {
                            lv[j] = __fadd_rn(lv[j], dg[j]);
                            two_sum(hv[j], lv[j], hv[j], lv[j]);
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&rel_bar[g]);
                }
            } else {
#pragma unroll
                for (int cb = 0; cb < kPartCols; cb += CB1) {
                    float d[NG][CB1];
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (g < ng_used) {
                            tmem_ld8(lane_addr + g * NT + cbase + cb, d[g]);
                        } else {
#pragma unroll
                            for (int j = 0; j < CB1; ++j) d[g][j] = 0.f;
                        }
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < CB1; ++j) sum_panel_groups<NG>(d, j, hv[cb + j], lv[cb + j]);
                }
                // tensor memory is free for the next tile's MMAs
                tc_fence_before();
                mbar_arrive(&tempty_bar[0]);
            }
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
                // tile i - NBUF (the group-wise release: group by group, in the first stage)
                const int buf = i % NBUF;
                if (!kGroupwise && i >= NBUF && !mbar_wait(&tempty_bar[buf], ((i / NBUF) - 1) & 1, &abort_flag)) {
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
                    if (kGroupwise && kc == 0) {
                        if (!issue_first_stage_er<NG, NT, kBBytes>(ns, i, tbase, ad0, bd0, idesc, rel_bar,
                                                                   &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                    } else {
                        issue_stage_ns<NG, NT, kBBytes>(ns, kc == 0, tbase + buf * NG * NT, ad0, bd0, idesc);
                    }
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
                        sum_panel_groups<NG>(d, j, h, l);
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

}  // namespace

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

cudaError_t launch_gemm_update_fused(const MixedBatch& b, int J, cudaStream_t s) {
    const int m = b.nt - J - 2;
    if (m <= 0) return cudaSuccess;
    if (b.update_tile == 64) return launch_gemm<1, 64, 4>(b, J, m * (m + 1), b.s, s, 2);
    return launch_update128(b, J, m * (m + 1) / 2, b.s, s, 2);
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

}  // namespace gp
