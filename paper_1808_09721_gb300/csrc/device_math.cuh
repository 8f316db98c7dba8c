// device_math.cuh -- scalar helpers shared by the kernels of this library.
//
// On GB300 an FP64 lane-op costs about 67 FP32 lane-ops of throughput, and the
// IEEE FP64 divide and square root cost ~7.5 FP64 ops each. The FP64 helpers
// here therefore start from the hardware's approximate reciprocal /
// reciprocal square root (rcp.approx.ftz.f64, rsqrt.approx.ftz.f64, one FP64
// op each) and refine with Newton's iteration for 1/x and 1/sqrt(x), which
// doubles the number of correct bits per step; two steps reach FP64 round-off
// from the approximation. The FP32 helpers use the SFU approximations
// directly: FP32 results only ever seed an FP64 refinement.
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

// 1/x: Newton's iteration y <- y + y (1 - x y), twice.
__device__ __forceinline__ double s_rcp(double x) {
    double y = approx_rcp(x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
// 1/x with a single Newton step (relative error ~ square of the approximation's).
__device__ __forceinline__ double s_rcp1(double x) {
    double y = approx_rcp(x);
    double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
// 1/sqrt(x): Newton's iteration y <- y + (y/2)(1 - x y^2), twice.
__device__ __forceinline__ double s_rsqrt(double x) {
    double y = approx_rsqrt(x);
    double h = 0.5 * y;
    double e = fma(-x * y, y, 1.0);
    y = fma(h, e, y);
    h = 0.5 * y;
    e = fma(-x * y, y, 1.0);
    return fma(h, e, y);
}

__device__ __forceinline__ float s_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float s_rcp1(float x) { return s_rcp(x); }
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
template <class T> __device__ __forceinline__ Dual<T> s_rcp1(Dual<T> a) { return s_rcp(a); }
template <class T> __device__ __forceinline__ Dual<T> s_rsqrt(Dual<T> a) {
    T y = s_rsqrt(a.v);
    return Dual<T>(y, T(-0.5) * a.d * y * y * y);
}
template <class T> __device__ __forceinline__ T value(T a) { return a; }
template <class T> __device__ __forceinline__ T value(Dual<T> a) { return a.v; }

// fused multiply-add that also works for duals
__device__ __forceinline__ double s_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float s_fma(float a, float b, float c) { return fmaf(a, b, c); }
template <class T> __device__ __forceinline__ Dual<T> s_fma(Dual<T> a, Dual<T> b, Dual<T> c) { return a * b + c; }

} // namespace rmhd
