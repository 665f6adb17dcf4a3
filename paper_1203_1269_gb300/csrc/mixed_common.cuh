// mixed_common.cuh -- what the split-precision kernels (k_mixed.cu, k_gemm.cu)
// share: the bf16 image layout of the operand slices, the tensor-memory,
// mbarrier and bulk-copy PTX, and the per-instance buffer addressing.
// Everything here is file-local (an anonymous namespace) to each including
// translation unit.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kChunkElems = GP_NB * 32;       // bf16 elements in one 128 x 32 image chunk
constexpr uint32_t kChunkBytes = kChunkElems * 2;
constexpr int kChunks = GP_NB / 32;           // 4 chunks per 128-wide panel
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

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

}  // namespace

}  // namespace gp
