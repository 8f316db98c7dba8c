// kernels_selftest.cu -- elementwise evaluation of the device arithmetic
// helpers the kernels are built on (approximate FP64 reciprocal, quotient and
// reciprocal square root with series refinement; FP64 <-> FP32 conversions on
// the integer pipes), so that their error bounds can be tested directly
// against IEEE arithmetic instead of only through whole-step parity.
#include <cuda_runtime.h>

#include "../../include/rmhd.h"
#include "device_math.cuh"

namespace {

__global__ void k_eval_math(int which, long long n, const double *x, const double *a, double *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        double r;
        switch (which) {
        case RMHD_MATH_RCP: r = rmhd::s_rcp(v); break;
        case RMHD_MATH_RSQRT: r = rmhd::s_rsqrt(v); break;
        case RMHD_MATH_DIV1: r = rmhd::s_div1(a[i], v); break;
        case RMHD_MATH_F32: r = (double)rmhd::f32_of(v); break;
        default: r = rmhd::f64_of((float)v); break;  // RMHD_MATH_F64: v is an FP32 value
        }
        out[i] = r;
    }
}

} // namespace

extern "C" int rmhd_eval_math(int which, long long n, const double *x, const double *a, double *out,
                              void *cuda_stream) {
    if (which < RMHD_MATH_RCP || which > RMHD_MATH_F64 || n < 0 || (n > 0 && (!x || !out)) ||
        (which == RMHD_MATH_DIV1 && n > 0 && !a))
        return RMHD_ERR_INVALID;
    if (n == 0) return RMHD_OK;
    if (cudaPeekAtLastError() != cudaSuccess) return RMHD_ERR_CUDA;
    const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_eval_math<<<(int)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(which, n, x, a, out);
    return cudaGetLastError() == cudaSuccess ? RMHD_OK : RMHD_ERR_CUDA;
}
