// ffloat.cuh -- float-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits (relative rounding ~2^-47 per operation).
//
// On GB300 the FP32 pipes issue 64 times as many lane-ops per clock as the
// FP64 pipe, so an operation built from the error-free transformations
// below (7-20 FP32 ops) costs several times less than one FP64 op. The flux
// kernels use it as their arithmetic type in the float-float precision mode;
// staging converts the FP64 state in, the epilogue converts the face-flux
// differences back to FP64 for the update.
//
// Error-free transformations (published methods, written out here):
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, 6 adds;
//   FastTwoSum (Dekker 1971): the same in 3 adds when |a| >= |b|;
//   TwoProduct with FMA: p + e = a b exactly, e = fma(a, b, -p).
// Addition is the "sloppy" float-float sum (TwoSum of the high parts, the low
// parts added to the error, FastTwoSum to renormalise); its error is bounded
// relative to |a| + |b|, which is what the differences of neighbouring cells
// in the reconstruction need. Multiplication keeps the hi*lo cross terms and
// drops lo*lo. Division takes the FP32 approximate reciprocal y of the
// divisor's high part and two correction steps, q1 = a_hi y and
// q2 = (a - x q1) y, for a relative error ~2^-44.
//
// __fadd_rn / __fmul_rn keep the compiler from contracting the steps into
// FMAs (that would break the exactness the transformations rely on). The
// range is FP32's: magnitudes above ~3e38 overflow to infinity and the
// low parts of magnitudes below ~1e-31 lose bits to underflow.
#pragma once
#include "device_math.cuh"

namespace rmhd {

struct ff {
    float hi, lo;
    ff() = default;
    __device__ __forceinline__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    // nearest float-float of a double (the residual x - hi is exact in FP64)
    __device__ __forceinline__ explicit ff(double x) : hi(f32_of(x)), lo(f32_of(x - f64_of(f32_of(x)))) {}
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return ff(s, e);
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff(s, __fadd_rn(b, -__fadd_rn(s, -a)));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator+(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }

// a b = p + e with p = fl(a_hi b_hi); e collects the exact product error and
// the cross terms
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a b + c with one renormalisation
__device__ __forceinline__ ff s_fma(ff a, ff b, ff c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const ff s = two_sum(p, c.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// 2 a + b: the doubling is exact, so one float-float sum
__device__ __forceinline__ ff s_fma2(ff a, ff b) { return ff(2.f * a.hi, 2.f * a.lo) + b; }
// a / x (x > 0 and normal in FP32 where this is used)
__device__ __forceinline__ ff s_div1(ff a, ff x) {
    const float y = s_rcp(x.hi);
    const float q1 = __fmul_rn(a.hi, y);
    const float p = __fmul_rn(x.hi, q1);  // x q1 = p + pe (to the cross term)
    float pe = fmaf(x.hi, q1, -p);
    pe = fmaf(x.lo, q1, pe);
    const float r = __fadd_rn(__fadd_rn(__fadd_rn(a.hi, -p), -pe), a.lo);  // a - x q1 (a_hi - p is exact)
    return fast_two_sum(q1, __fmul_rn(r, y));
}

template <> __device__ __forceinline__ ff to_t<ff>(double x) { return ff(x); }
__device__ __forceinline__ double to_f64(ff a) { return f64_of(a.hi) + f64_of(a.lo); }

} // namespace rmhd
