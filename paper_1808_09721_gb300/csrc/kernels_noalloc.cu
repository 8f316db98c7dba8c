// kernels_noalloc.cu -- a diagnostics reduction that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool or
// arena owns the whole device, a host framework that forbids allocation after
// start-up, or a caller inside a region where allocation would synchronise the
// device. rmhd_diagnostics_noalloc serves them: it computes the same numbers
// as rmhd_diagnostics (cell sums of D, tau, S_x, B_x and the charge variable
// times the cell volume, max |v|, count of non-finite conserved values) from
// caller-provided device arrays of a 1-D, 2-D or 3-D grid, and keeps its
// partial sums in the file-scope device array below instead of in any
// allocated workspace.
//
// The scratch array is a device global: every GPU that loads this library
// holds its 512 KiB until the process exits. It holds one 8-double partial per
// block of 2048 cells, so inputs are limited to 8192 x 2048 = 16,777,216 cells.
// All calls share it and it keeps the last call's contents; each call writes
// every partial it later reads, so nothing needs clearing, but two calls whose
// kernels overlap on the GPU (different streams, no ordering) race on it.
// The device address of the array is looked up once per device and cached for
// the life of the process; a cudaDeviceReset reloads the module (possibly at
// another address), so this call must not be used on a device after a reset.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rmhd.h"

namespace {

constexpr int kCellsPerBlock = 2048;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;
constexpr long long kMaxCells = (long long)kMaxBlocks * kCellsPerBlock;
constexpr int kMaxDevices = 64;

// In host code this name is a host-side stand-in, not a device address: the
// host must obtain the address with cudaGetSymbolAddress (see scratch_ptr).
__device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 8];

std::mutex g_mutex;
double *g_ptr[kMaxDevices] = {nullptr};

// Per-device set-up, with that device current: look up the device address of
// the scratch array once and cache it.
cudaError_t scratch_ptr(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = (double *)p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

// Block b reduces cells [b * 2048, min((b + 1) * 2048, ncell)) into 8 partials.
__global__ void __launch_bounds__(kThreads) k_partials(int model, long long ncell, const double *cons,
                                                       const double *prims, double *partials) {
    const int nc = model == 0 ? 14 : 18;
    const int iT = 4, iS = 1, iB = model == 0 ? 5 : 10, iR = model == 0 ? 11 : 5;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long c0 = (long long)blockIdx.x * kCellsPerBlock;
    const long long c1 = c0 + kCellsPerBlock < ncell ? c0 + kCellsPerBlock : ncell;
    for (long long c = c0 + threadIdx.x; c < c1; c += kThreads) {
        acc[0] += cons[0 * ncell + c];
        acc[1] += cons[iT * ncell + c];
        acc[2] += cons[iS * ncell + c];
        acc[3] += cons[iB * ncell + c];
        acc[4] += cons[iR * ncell + c];
        for (int s = 0; s < (model == 0 ? 1 : 2); ++s) {
            double vx = prims[(5 * s + 1) * ncell + c], vy = prims[(5 * s + 2) * ncell + c],
                   vz = prims[(5 * s + 3) * ncell + c];
            acc[5] = fmax(acc[5], sqrt(vx * vx + vy * vy + vz * vz));
        }
        double bad = 0.0;
        for (int v = 0; v < nc; ++v) bad += isfinite(cons[v * ncell + c]) ? 0.0 : 1.0;
        acc[6] += bad;
    }
    __shared__ double red[8][kThreads];
    for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 8; ++k)
                red[k][threadIdx.x] = k == 5 ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + off])
                                             : red[k][threadIdx.x] + red[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

// One block combines the partials in a fixed order and scales the sums.
__global__ void __launch_bounds__(kThreads) k_combine(int nblocks, double vol, const double *partials, double *out) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int k = 0; k < 8; ++k) acc[k] = k == 5 ? fmax(acc[k], partials[b * 8 + k]) : acc[k] + partials[b * 8 + k];
    __shared__ double red[8][kThreads];
    for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 8; ++k)
                red[k][threadIdx.x] = k == 5 ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + off])
                                             : red[k][threadIdx.x] + red[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) out[k] = red[k][0] * vol;
        out[5] = red[5][0];
        out[6] = red[6][0];
    }
}

} // namespace

extern "C" int rmhd_diagnostics_noalloc(int model, int nx, int ny, int nz, double dx, double dy, double dz,
                                        const double *cons, const double *prims, double *out, void *cuda_stream) {
    if ((model != RMHD_RESISTIVE && model != RMHD_TWO_FLUID) || nx < 1 || ny < 1 || nz < 1 || !cons || !prims ||
        !out || !(dx > 0.0) || (ny > 1 && !(dy > 0.0)) || (nz > 1 && (ny < 2 || !(dz > 0.0))))
        return RMHD_ERR_INVALID;
    const long long ncell = (long long)nx * ny * nz;
    if (ncell > kMaxCells) return RMHD_ERR_NOMEM;  // beyond the static scratch
    // an error left pending by earlier work on this thread is not this call's:
    // report it without clearing it and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return RMHD_ERR_CUDA;
    double *partials = nullptr;
    if (scratch_ptr(&partials) != cudaSuccess) return RMHD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nblocks = (int)((ncell + kCellsPerBlock - 1) / kCellsPerBlock);
    const double vol = dx * (ny > 1 ? dy : 1.0) * (nz > 1 ? dz : 1.0);
    k_partials<<<nblocks, kThreads, 0, s>>>(model, ncell, cons, prims, partials);
    if (cudaGetLastError() != cudaSuccess) return RMHD_ERR_CUDA;  // this launch's own error
    k_combine<<<1, kThreads, 0, s>>>(nblocks, vol, partials, out);
    if (cudaGetLastError() != cudaSuccess) return RMHD_ERR_CUDA;
    return RMHD_OK;
}
