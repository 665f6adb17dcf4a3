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

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) { return df_fma(a, b, dfl{0.f, 0.f}); }

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

}  // namespace gp
