// slices.cuh -- cutting double-float rows into the bf16 slices that the
// split GEMMs read (the factorisation's panels in k_mixed.cu, the kriging
// variance's operands in k_var_tc.cu): a row scaled by 2^(7 - E), E the
// exponent of its largest high word, is cut into s slices q_a 2^(-8a),
// |q_a| <= 128, each exact in bf16 (after Ozaki, Ogita, Oishi & Rump 2012),
// and written into the 64-byte swizzled image chunks of mixed_common.cuh.
// File-local (an anonymous namespace) to each including translation unit.
#pragma once

#include "mixed_common.cuh"

namespace gp {

namespace {

// exponent E of a row maximum mx = f 2^E, f in [0.5, 1) (0 for mx == 0): the
// slices of the row are cut from x 2^(7 - E), whose magnitude is below 128
__device__ __forceinline__ int exponent_of(float mx) {
    if (mx == 0.f) return 0;
    const int bits = __float_as_int(mx);
    const int be = (bits >> 23) & 0xff;
    if (be != 0) return be - 126;
    int E;
    frexpf(mx, &E);
    return E;
}

// 2^(7 - E) as two exact float factors (7 - E may leave the float range)
__device__ __forceinline__ void slice_scale(int E, float& sa, float& sb) {
    const int e2 = 7 - E;
    const int ea = e2 > 127 ? 127 : (e2 < -126 ? -126 : e2);
    const int eb = e2 - ea;
    sa = __int_as_float((ea + 127) << 23);
    sb = (eb == 0) ? 1.f : __int_as_float(((eb > 127 ? 127 : (eb < -126 ? -126 : eb)) + 127) << 23);
}

// One 256-bit store (two adjacent 16-byte pieces, 32-byte aligned).
__device__ __forceinline__ void st_global_v8(void* p, uint4 a, uint4 b) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
                 "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}

// Slices of 8 values (one 16-byte piece per slice): m = the slice's values.
__device__ __forceinline__ uint4 next_slice8(float (&xh)[8], float (&xl)[8], float w) {
    float m[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float qv = rintf(xh[e]);
        m[e] = __fmul_rn(qv, w);
        two_sum(__fsub_rn(xh[e], qv), xl[e], xh[e], xl[e]);
        xh[e] = __fmul_rn(xh[e], 256.f);
        xl[e] = __fmul_rn(xl[e], 256.f);
    }
    uint4 pk;
    pk.x = pack_bf16x2(m[0], m[1]);
    pk.y = pack_bf16x2(m[2], m[3]);
    pk.z = pack_bf16x2(m[4], m[5]);
    pk.w = pack_bf16x2(m[6], m[7]);
    return pk;
}

// Slices of one thread's NC values of row r (columns k0 .. k0 + NC - 1 of
// image chunk `chunk0`, k0 = 0, 8, 16 or 24; slice a at chunk0 + a *
// slice_bytes): NC / 8 pieces of 8.  With NC = 16 (k0 = 0 or 16) the two
// pieces of a slice occupy one aligned 32-byte sector of the row (the
// swizzle only swaps them), written by one 256-bit store.
template <int NC>
__device__ __forceinline__ void slice_pieces(const float2 (&v)[NC], float sa, float sb, int r, int k0,
                                             int ns, uint8_t* chunk0, size_t slice_bytes) {
    static_assert(NC == 8 || NC == 16, "one or two pieces per thread");
    float xh[NC / 8][8], xl[NC / 8][8];
#pragma unroll
    for (int h = 0; h < NC / 8; ++h)
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            xh[h][e] = __fmul_rn(__fmul_rn(v[8 * h + e].x, sa), sb);
            xl[h][e] = __fmul_rn(__fmul_rn(v[8 * h + e].y, sa), sb);
        }
    const uint32_t off0 = image_piece(r, k0);
    const uint32_t off1 = (NC == 16) ? image_piece(r, k0 + 8) : off0;
    float w = 1.f;
#pragma unroll
    for (int a = 0; a < GP_MAX_SLICES; ++a) {
        if (a >= ns) break;
        uint8_t* base = chunk0 + (size_t)a * slice_bytes;
        const uint4 p0 = next_slice8(xh[0], xl[0], w);
        if (NC == 16) {
            const uint4 p1 = next_slice8(xh[NC / 8 - 1], xl[NC / 8 - 1], w);
            if (off0 < off1) st_global_v8(base + off0, p0, p1);
            else             st_global_v8(base + off1, p1, p0);
        } else {
            *reinterpret_cast<uint4*>(base + off0) = p0;
        }
        w = __fmul_rn(w, 0.00390625f);
    }
}

}  // namespace

}  // namespace gp
