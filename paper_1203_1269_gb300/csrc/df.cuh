// df.cuh -- double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On this GPU an FP64 instruction costs about 64
// FP32 instructions, so the split-precision path keeps its working matrix,
// its combination of tensor-core partial sums and its solves in this form.
//
// The error-free transformations are the published ones: TwoSum (D. Knuth,
// TAOCP vol. 2), FastTwoSum (T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971) and the exact
// product through a fused multiply-add.  The _rn intrinsics keep the compiler
// from contracting or reordering them.
#pragma once

#include <cuda_runtime.h>

namespace gp {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl df_make(float hi, float lo) {
    dfl r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return {s, e};
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// c + a * b
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, e));
    fast_two_sum(s, t, s, t);
    return {s, t};
}

// c - a * b
__device__ __forceinline__ dfl df_fms(dfl a, dfl b, dfl c) { return df_fma(df_neg(a), b, c); }

// a * b: the exact product of the high words, its error and the cross terms
// (what df_fma gives with c = 0, without the additions of zero)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    fast_two_sum(p, e, s, t);
    return {s, t};
}

// a / b to about 46 bits: one Newton correction of the float quotient
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfl r = df_fms(dfl{q1, 0.f}, b, a);      // a - q1 b
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_make(q1, q2);
}

__device__ __forceinline__ dfl df_from_double(double v) {
    const float h = __double2float_rn(v);
    const float l = __double2float_rn(v - (double)h);
    return {h, l};
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfl df_load(const float2* p) {
    const float2 v = *p;
    return {v.x, v.y};
}

__device__ __forceinline__ void df_store(float2* p, dfl a) { *p = make_float2(a.hi, a.lo); }

// Entries of the table of 2^(-j/N) that df_exp_neg reads (N = 1024: 8 KB
// of double-float values in shared memory).
constexpr int kExpTabBits = 10;
constexpr int kExpTab = 1 << kExpTabBits;

// exp(-S) to about 46 bits, after P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15 (1989), with a table of N = 1024 entries:
//   k = round(S N / ln 2),  r = S - k ln2/N  (|r| <= ln2/(2N) = 3.4e-4, a
//   Cody-Waite reduction with ln2/N held as two floats),
//   exp(-S) = 2^(-k/N) exp(-r),  2^(-k/N) = 2^(-m) tab[j] for k = N m + j,
//   exp(-r) = 1 - r + q,  q = r^2/2 - r^3/6 (the r^4 term is below 2^-50).
// q < 6e-8 is needed to float precision only, so past the reduction the
// only double-float steps are 1 - r and the product with the table.  S may
// be negative down to -83 (the logarithms of df_log's Newton step).
// tab[j] = 2^(-j/N) as double-float (filled by fill_exp2_table).  Results
// below 2^-125 (S > 86.6) are returned as zero.
__device__ __forceinline__ dfl df_exp_neg(dfl S, const dfl* tab) {
    constexpr double kLn2OverN = 0.693147180559945309417232121458176568 / kExpTab;
    constexpr float kCHi = (float)kLn2OverN;
    constexpr float kCLo = (float)(kLn2OverN - (double)kCHi);
    constexpr float kNOverLn2 = (float)(kExpTab / 0.693147180559945309417232121458176568);
    if (!(S.hi < 86.6f)) return {0.f, 0.f};
    const float kf = rintf(__fmul_rn(S.hi, kNOverLn2));
    const int k = (int)kf;
    // r = S - k (C_hi + C_lo); k C_hi as p1 + e1 exactly
    const float p1 = __fmul_rn(kf, kCHi);
    const float e1 = __fmaf_rn(kf, kCHi, -p1);
    const float p2 = __fmul_rn(kf, kCLo);
    float rh = __fsub_rn(S.hi, p1);   // exact: p1 is within a factor 2 of S.hi, or 0
    float rl = __fsub_rn(__fsub_rn(S.lo, e1), p2);
    two_sum(rh, rl, rh, rl);
    // q = rh^2/2 - rh^3/6 + rh rl  (r^2/2 to first order in rl)
    float q = __fmaf_rn(rh, -1.f / 6.f, 0.5f);
    q = __fmaf_rn(rh, q, rl);
    q = __fmul_rn(rh, q);
    float s, t;
    fast_two_sum(1.f, -rh, s, t);     // |rh| < 1
    t = __fadd_rn(__fsub_rn(t, rl), q);
    fast_two_sum(s, t, s, t);
    dfl e = df_mul(dfl{s, t}, tab[k & (kExpTab - 1)]);
    const float sc = __int_as_float((127 - (k >> kExpTabBits)) << 23);   // 2^-m, -120 <= m <= 125
    e.hi = __fmul_rn(e.hi, sc);
    e.lo = __fmul_rn(e.lo, sc);
    return e;
}

// ln x for x > 0 (x in [2^-60, 2^60]): a float seed y0 = logf(x) and one
// Newton step y = y0 + x exp(-y0) - 1 in double-float, which doubles the
// seed's ~22 correct bits.
__device__ __forceinline__ dfl df_log(dfl x, const dfl* tab) {
    const float y0 = logf(x.hi);
    const dfl e = df_exp_neg(dfl{y0, 0.f}, tab);          // exp(-y0)
    const dfl t = df_fma(x, e, dfl{-1.f, 0.f});            // x exp(-y0) - 1
    return df_add(dfl{y0, 0.f}, t);
}

// Exponent modes of |d|^p: the two exact cases and the general one.
enum : int { kPowGeneral = 0, kPowOne = 1, kPowTwo = 2 };

__host__ __device__ __forceinline__ int pow_mode(double p) {
    return p == 2.0 ? kPowTwo : (p == 1.0 ? kPowOne : kPowGeneral);
}

// |d|^p for p in (0, 2] as exp(p ln |d|) in double-float (pd = p as
// double-float).  |d| outside [2^-60, 2^60] (far from any realistic
// coordinate difference) takes the double pow instead, with the result
// clamped to [0, 2^120] so that a zero theta still gives a zero term.
__device__ __forceinline__ dfl df_powabs(dfl d, int mode, double p, dfl pd, const dfl* tab) {
    if (d.hi < 0.f) d = df_neg(d);
    if (d.hi == 0.f) return {0.f, 0.f};
    if (!(d.hi >= 0x1p-60f && d.hi <= 0x1p60f)) {
        const double a = df_to_double(d);
        const double v = (mode == kPowTwo) ? a * a : (mode == kPowOne ? a : pow(a, p));
        return df_from_double(fmin(v, 0x1p120));
    }
    if (mode == kPowTwo) return df_mul(d, d);
    if (mode == kPowOne) return d;
    return df_exp_neg(df_neg(df_mul(pd, df_log(d, tab))), tab);
}

// tab[j] = 2^(-j/N), j = 0 .. N - 1, as double-float (the block's threads in
// turn; the caller synchronises before the table is read).
__device__ __forceinline__ void fill_exp2_table(dfl* tab) {
    for (int j = threadIdx.x; j < kExpTab; j += blockDim.x)
        tab[j] = df_from_double(exp2(-(double)j / (double)kExpTab));
}

}  // namespace gp
