// device_math.cuh -- scalar helpers shared by the kernels of this library.
//
// On GB300 an FP64 lane-op costs about 67 FP32 lane-ops of throughput, and the
// IEEE FP64 divide and square root cost ~7.5 FP64 ops each. The FP64 helpers
// here therefore start from the hardware's approximate reciprocal /
// reciprocal square root (rcp.approx.ftz.f64, rsqrt.approx.ftz.f64: one FP64
// op each, relative error below 2^-19 as measured on GB300) and refine with
// the truncated series of 1/(1 - e) and (1 - e)^(-1/2) in the residual
// e = 1 - x y0 (resp. 1 - x y0^2): the second-order terms leave an O(e^3)
// ~ 2^-57 relative error, FP64 round-off, in 3 (resp. 4) FP64 ops. The FP32
// helpers use the SFU approximations directly: FP32 results only ever seed
// an FP64 refinement.
#pragma once
#include <cuda_runtime.h>

namespace rmhd {

__device__ __forceinline__ double approx_rcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}
__device__ __forceinline__ double approx_rsqrt(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x = y0 / (1 - e) with e = 1 - x y0:  y0 (1 + e + e^2) + O(e^3).
__device__ __forceinline__ double s_rcp(double x) {
    double y = approx_rcp(x);
    double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
// a/x with a single Newton step: with t = a y0 and e = 1 - x y0, a/x = t/(1 - e)
// ~ t (1 + e); relative error ~e^2 ~ 2^-38 in 3 FP64 ops after the approximation.
__device__ __forceinline__ double s_div1(double a, double x) {
    double y = approx_rcp(x);
    double t = a * y;
    double e = fma(-x, y, 1.0);
    return fma(t, e, t);
}
// 1/sqrt(x) = y0 (1 - e)^(-1/2) with e = 1 - x y0^2:  y0 (1 + e/2 + 3 e^2/8) + O(e^3).
__device__ __forceinline__ double s_rsqrt(double x) {
    double y = approx_rsqrt(x);
    double e = fma(-x * y, y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

// Conversions between FP64 and FP32 on the integer pipes. The conversion
// instructions run on the FP64 pipe, the one this library is bound by; these
// use shifts and logic ops instead (both pipes idle in the FP64-bound kernels).
//
// f32_of: round to nearest (ties away from zero) on the first dropped bit,
// FP32 subnormals included; magnitudes above the FP32 range (and infinities,
// NaNs) give a signed infinity.
__device__ __forceinline__ float f32_of(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // FP32 biased exponent
    const unsigned m = __funnelshift_l(lo, hi, 3) & 0x7fffffu, g = (lo >> 28) & 1u;
    unsigned mag = (((unsigned)e << 23) | m) + g;
    if (e <= 0) {  // FP32 subnormal range: shift the 24-bit significand down, then round
        const unsigned t = 0x1000000u | (m << 1) | g;
        mag = e < -23 ? 0u : ((t >> (1 - e)) + 1u) >> 1;
    }
    if (e >= 255) mag = 0x7f800000u;
    return __uint_as_float(sign | mag);
}
// f64_of: exact for every FP32 value (subnormals normalised; infinities and
// NaNs kept).
__device__ __forceinline__ double f64_of(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 255u) hi |= 0x7ff00000u;
    if (e == 0u) {  // zero or subnormal: m * 2^-149
        const int s = __clz(m) - 8;  // shift that puts the leading bit at 23
        const unsigned mn = (m << s) & 0x7fffffu;
        hi = m ? (sign | ((unsigned)(897 - s) << 20) | (mn >> 3)) : sign;
        lo = m ? (mn << 29) : 0u;
    }
    return __hiloint2double((int)hi, (int)lo);
}
// conversions to and from a flux arithmetic type T (identity for double)
template <class T> __device__ __forceinline__ T to_t(double x) { return x; }
template <> __device__ __forceinline__ float to_t<float>(double x) { return f32_of(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f64_of(x); }

__device__ __forceinline__ float s_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float s_div1(float a, float x) { return a * s_rcp(x); }
__device__ __forceinline__ float s_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Forward-mode dual number: value and one directional derivative. Used to
// build Jacobian columns of the implicit-stage residual exactly (up to the
// arithmetic's rounding) from the same code that evaluates the residual.
template <class T>
struct Dual {
    T v, d;
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T a) : v(a), d(T(0)) {}
    __device__ __forceinline__ Dual(T a, T b) : v(a), d(b) {}
};
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return Dual<T>(a * b.v, a * b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return Dual<T>(a.v * b, a.d * b); }
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return Dual<T>(a.v + b, a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return Dual<T>(a + b.v, b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return Dual<T>(a.v - b, a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return Dual<T>(a - b.v, -b.d); }
template <class T> __device__ __forceinline__ Dual<T> s_rcp(Dual<T> a) { T r = s_rcp(a.v); return Dual<T>(r, -a.d * r * r); }
template <class T> __device__ __forceinline__ Dual<T> s_rsqrt(Dual<T> a) {
    T y = s_rsqrt(a.v);
    return Dual<T>(y, T(-0.5) * a.d * y * y * y);
}
template <class T> __device__ __forceinline__ T value(T a) { return a; }
template <class T> __device__ __forceinline__ T value(Dual<T> a) { return a.v; }

// fused multiply-add that also works for duals
__device__ __forceinline__ double s_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float s_fma(float a, float b, float c) { return fmaf(a, b, c); }
// 2 a + b (one rounding in FP64 and FP32)
__device__ __forceinline__ double s_fma2(double a, double b) { return fma(2.0, a, b); }
__device__ __forceinline__ float s_fma2(float a, float b) { return fmaf(2.f, a, b); }
template <class T> __device__ __forceinline__ Dual<T> s_fma(Dual<T> a, Dual<T> b, Dual<T> c) { return a * b + c; }

} // namespace rmhd
