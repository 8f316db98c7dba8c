// kernels_stage.cu -- per-cell kernels: the implicit IMEX stage solve (Eq.
// implicit stage of Wright & Hawke, arXiv:1808.09721), primitive <-> conserved
// maps (Eq. resistive prims, Eq. twoFluid cons), primitive recovery
// (Sec. 2.1.3), layout packing and the diagnostics reduction.
#include "rmhd_internal.h"
#include "physics_sf.cuh"
#include "physics_tf.cuh"

namespace rmhd {

static constexpr int kStageThreads = 128;
static constexpr int kNRef = 2;  // FP64 refinement passes per stage solve

// The status word is one 64-bit key (cell << 8 | -code), initialised to all
// ones; atomicMin keeps the smallest failing cell together with its own code.
__device__ __forceinline__ void record(int *status, int st, long long cell) {
    if (st != 0)
        atomicMin(reinterpret_cast<unsigned long long *>(status),
                  ((unsigned long long)cell << 8) | (unsigned long long)((-st) & 0xff));
}

__device__ __forceinline__ int wrap(int i, int n, int bc) {
    if (bc == 1) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Restart list: rlist[0] = number of cells, rlist[1] = restart blocks done,
// rlist[2 ..] = cells. A cell whose first start failed goes to the list (or,
// beyond its capacity, is reported as failed).
__device__ __forceinline__ void defer_or_record(const StageArgs &a, int st, long long cell) {
    if (st == sf::ST_NEWTON && a.rlist) {
        const int slot = atomicAdd(a.rlist, 1);
        if (slot < a.rcap) {
            a.rlist[2 + slot] = (int)cell;
            return;
        }
    }
    record(a.status, st, cell);
}

// End of a restart kernel: the last block to finish (every block has read
// the count by then) empties the list for the next stage.
__device__ __forceinline__ void restart_done(int *rlist) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&rlist[1], 1) == (int)gridDim.x - 1) {
            rlist[0] = 0;
            rlist[1] = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------- stage
// 5 blocks per SM (at most 96 registers): the solve is latency-bound, and
// 20 warps per SM hide more of its FP64 and MUFU latency than 16 (no spills)
// STATS: instantiation that also fills the iteration histogram a.hist
template <bool STATS>
__global__ void __launch_bounds__(kStageThreads, 5) k_stage_sf(Grid g, Phys ph, StageArgs a, double cpsi) {
    using namespace sf;
    sf::StageConst k{a.adt, cpsi, ph.sigma, ph.gamma, a.maxpass > 0 ? a.maxpass : 8, a.hist};
    const long long c0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, cs = (long long)gridDim.x * blockDim.x;
    if (a.first_start != 0) {  // test control: every cell begins at a later start
        for (long long cell = c0; cell < g.ncell; cell += cs) defer_or_record(a, sf::ST_NEWTON, cell);
        return;
    }
    for (long long cell = c0; cell < g.ncell; cell += cs) {
        const double pw = a.wwarm[P * g.plane + cell];
        const int st = stage_solve<kNRef, STATS>(a.r + cell, g.plane, pw, k, a.q + cell, a.w + cell,
                                                 a.src ? a.src + cell : nullptr);
        defer_or_record(a, st, cell);
    }
}

// The listed cells again, from the ideal-limit start and then along a
// continuation in a dt (physics_sf.cuh: stage_restarts). Launched after every
// single-fluid stage kernel; with an empty list every thread exits at once
// (measured: ~4 us per step inside the step's CUDA graph, where an in-kernel
// tail run by the stage kernel's last block cost ~20 us).
template <bool STATS>
__global__ void k_restart_sf(Grid g, Phys ph, StageArgs a, double cpsi) {
    using namespace sf;
    const int n = min(*(volatile int *)a.rlist, a.rcap);
    sf::StageConst k{a.adt, cpsi, ph.sigma, ph.gamma, a.maxpass > 0 ? a.maxpass : 8, a.hist};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long cell = a.rlist[2 + e];
        const double pw = a.wwarm[P * g.plane + cell];
        record(a.status,
               stage_restarts<kNRef, STATS>(a.r + cell, g.plane, pw, k, a.q + cell, a.w + cell, a.first_start,
                                            a.src ? a.src + cell : nullptr),
               cell);
    }
    restart_done(a.rlist);
}

// Two fluids: the 7 x 7 Jacobian of each thread and its LU factors live in a
// strided slice of shared memory (not in local memory: the pivoted
// factorisation indexes it with run-time rows).
static constexpr int kStageThreadsTF = 64;
// 8 blocks per SM (at most 128 registers, a 32-byte spill): 16 warps per SM
// instead of 8 hide the latency of the 7-unknown solve (measured 18% faster)
template <bool STATS>
__global__ void __launch_bounds__(kStageThreadsTF, 8) k_stage_tf(Grid g, Phys ph, StageArgs a, double cpsi) {
    using namespace tf;
    __shared__ float sJ[49 * kStageThreadsTF];
    const Mat Jm{sJ + threadIdx.x, kStageThreadsTF};
    tf::StageConst k{a.adt, cpsi, a.maxpass > 0 ? a.maxpass : 8, a.hist};
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        const int st =
            stage_solve<kNRef, STATS>(a.r + cell, g.plane, a.wwarm + cell, k, ph, a.q + cell, a.w + cell, Jm,
                                      a.src ? a.src + cell : nullptr);
        record(a.status, st, cell);
    }
}

// restart kernels: a small fixed grid (the list is short: cells whose first start failed)
static constexpr int kRestartBlocks = 64;

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > (1 << 30) ? (1 << 30) : b));
}

cudaError_t launch_stage(int model, const Grid &g, const Phys &ph, const StageArgs &a, cudaStream_t s) {
    double cpsi = 1.0 / (1.0 + a.adt * ph.kappa);
    int blocks = grid_for(g.ncell, kStageThreads);
    const int btf = grid_for(g.ncell, kStageThreadsTF);
    if (model == 0) {
        if (a.hist) k_stage_sf<true><<<blocks, kStageThreads, 0, s>>>(g, ph, a, cpsi);
        else k_stage_sf<false><<<blocks, kStageThreads, 0, s>>>(g, ph, a, cpsi);
        if (a.rlist) {
            if (a.hist) k_restart_sf<true><<<kRestartBlocks, 64, 0, s>>>(g, ph, a, cpsi);
            else k_restart_sf<false><<<kRestartBlocks, 64, 0, s>>>(g, ph, a, cpsi);
        }
    } else {
        if (a.hist) k_stage_tf<true><<<btf, kStageThreadsTF, 0, s>>>(g, ph, a, cpsi);
        else k_stage_tf<false><<<btf, kStageThreadsTF, 0, s>>>(g, ph, a, cpsi);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched stage
// One thread per packed cell; the run's a_ii dt, 1/(1 + a_ii dt kappa) and
// conductivity come from the per-run tables.
// the block size is the autotuner's choice: cap registers as k_stage_sf's bounds do
template <bool STATS>
__global__ void __maxnreg__(96) k_stage_batch_sf(Grid g, Phys ph, StageArgs a, BatchArgs b) {
    using namespace sf;
    const long long c0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, cs = (long long)gridDim.x * blockDim.x;
    if (a.first_start != 0) {  // test control: every cell begins at a later start
        for (long long cell = c0; cell < g.ncell; cell += cs) defer_or_record(a, sf::ST_NEWTON, cell);
        return;
    }
    for (long long cell = c0; cell < g.ncell; cell += cs) {
        const int run = b.run_of[cell];
        sf::StageConst k{b.adt[run], b.cpsi[run], b.sigma[run], ph.gamma, a.maxpass > 0 ? a.maxpass : 8, a.hist};
        const int st =
            stage_solve<kNRef, STATS>(a.r + cell, g.plane, a.wwarm[P * g.plane + cell], k, a.q + cell, a.w + cell);
        defer_or_record(a, st, cell);
    }
}

template <bool STATS>
__global__ void k_restart_batch_sf(Grid g, Phys ph, StageArgs a, BatchArgs b) {
    using namespace sf;
    const int n = min(*(volatile int *)a.rlist, a.rcap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long cell = a.rlist[2 + e];
        const int run = b.run_of[cell];
        sf::StageConst k{b.adt[run], b.cpsi[run], b.sigma[run], ph.gamma, a.maxpass > 0 ? a.maxpass : 8, a.hist};
        record(a.status,
               stage_restarts<kNRef, STATS>(a.r + cell, g.plane, a.wwarm[P * g.plane + cell], k, a.q + cell, a.w + cell,
                                            a.first_start),
               cell);
    }
    restart_done(a.rlist);
}

template <bool STATS>
__global__ void k_stage_batch_tf(Grid g, Phys ph, StageArgs a, BatchArgs b) {
    using namespace tf;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        const int run = b.run_of[cell];
        Phys pr = ph;
        pr.sigma = b.sigma[run];
        pr.eta = b.eta[run];
        tf::StageConst k{b.adt[run], b.cpsi[run], a.maxpass > 0 ? a.maxpass : 8, a.hist};
        float jl[49];
        const int st = stage_solve<kNRef, STATS>(a.r + cell, g.plane, a.wwarm + cell, k, pr, a.q + cell, a.w + cell,
                                                 tf::Mat{jl, 1});
        record(a.status, st, cell);
    }
}

cudaError_t launch_stage_batch(int model, const Grid &g, const Phys &ph, const StageArgs &a, const BatchArgs &b,
                               int threads, cudaStream_t s) {
    int blocks = grid_for(g.ncell, threads);
    if (model == 0) {
        if (a.hist) k_stage_batch_sf<true><<<blocks, threads, 0, s>>>(g, ph, a, b);
        else k_stage_batch_sf<false><<<blocks, threads, 0, s>>>(g, ph, a, b);
        if (a.rlist) {
            if (a.hist) k_restart_batch_sf<true><<<kRestartBlocks, 64, 0, s>>>(g, ph, a, b);
            else k_restart_batch_sf<false><<<kRestartBlocks, 64, 0, s>>>(g, ph, a, b);
        }
    } else {
        if (a.hist) k_stage_batch_tf<true><<<blocks, threads, 0, s>>>(g, ph, a, b);
        else k_stage_batch_tf<false><<<blocks, threads, 0, s>>>(g, ph, a, b);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- prims -> cons
// user primitives are dense [np][nz][ny][nx]; the state uses padded planes.
__global__ void k_set_prims_sf(Grid g, Phys ph, const double *U, double *q, double *w, int *status) {
    using namespace sf;
    // cell counts are below 2^31 (validated), so 32-bit index arithmetic
    const long long n = g.ncell;
    const unsigned nxy = (unsigned)g.nx * (unsigned)g.ny;
    const double r2x = 2.0 * g.rdx4, r2y = 2.0 * g.rdy4, r2z = 2.0 * g.rdz4;  // 1 / (2 dx) ...
    const double hfac = ph.gamma / (ph.gamma - 1.0);
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        const unsigned c32 = (unsigned)cell;
        const int kz = (int)(c32 / nxy);
        const unsigned c2 = c32 - (unsigned)kz * nxy;  // index within the x-y plane
        const int j = (int)(c2 / (unsigned)g.nx), i = (int)(c2 - (unsigned)j * (unsigned)g.nx);
        const long long pz = (long long)kz * nxy;      // first cell of the plane
        double rho = U[0 * n + cell], v[3] = {U[1 * n + cell], U[2 * n + cell], U[3 * n + cell]}, p = U[4 * n + cell];
        double B[3] = {U[5 * n + cell], U[6 * n + cell], U[7 * n + cell]};
        double E[3] = {U[8 * n + cell], U[9 * n + cell], U[10 * n + cell]};
        double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        bool ok = rho > 0.0 && p > 0.0 && v2 < 1.0 && isfinite(rho + p + v2 + B[0] + B[1] + B[2] + E[0] + E[1] + E[2]);
        if (!ok) { record(status, -1, cell); continue; }
        // Gauss's law varrho = div E, central differences with the boundary map
        int il = wrap(i - 1, g.nx, g.bcx), ir = wrap(i + 1, g.nx, g.bcx);
        double divE = (U[8 * n + pz + (long long)j * g.nx + ir] - U[8 * n + pz + (long long)j * g.nx + il]) * r2x;
        if (g.ny > 1) {
            int jl = wrap(j - 1, g.ny, g.bcy), jr = wrap(j + 1, g.ny, g.bcy);
            divE += (U[9 * n + pz + (long long)jr * g.nx + i] - U[9 * n + pz + (long long)jl * g.nx + i]) * r2y;
        }
        if (g.nz > 1) {
            int kl = wrap(kz - 1, g.nz, g.bcz), kr = wrap(kz + 1, g.nz, g.bcz);
            divE += (U[10 * n + (long long)kr * nxy + c2] - U[10 * n + (long long)kl * nxy + c2]) * r2z;
        }
        double W = s_rsqrt(1.0 - v2);
        double h = fma(hfac * p, s_rcp(rho), 1.0);
        double Z = rho * h * W * W;
        double ExB[3];
        cross(E, B, ExB);
        double qc[NC];
        qc[D] = rho * W;
        for (int k = 0; k < 3; ++k) {
            qc[SX + k] = Z * v[k] + ExB[k];
            qc[BX + k] = B[k];
            qc[EX + k] = E[k];
        }
        qc[TAU] = Z - p + 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) - rho * W;
        qc[RHOE] = divE;
        qc[PSI] = 0.0;
        qc[PHI] = 0.0;
        for (int k = 0; k < NC; ++k) q[k * g.plane + cell] = qc[k];
        w[VX * g.plane + cell] = v[0];
        w[VY * g.plane + cell] = v[1];
        w[VZ * g.plane + cell] = v[2];
        w[P * g.plane + cell] = p;
        w[LOR * g.plane + cell] = W;
    }
}

__global__ void k_set_prims_tf(Grid g, Phys ph, const double *U, double *q, double *w, int *status) {
    using namespace tf;
    const long long n = g.ncell;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        double qc[NC];
        for (int k = 0; k < NC; ++k) qc[k] = 0.0;
        const double mu[2] = {ph.mu_e, ph.mu_p};
        double B[3] = {U[10 * n + cell], U[11 * n + cell], U[12 * n + cell]};
        double E[3] = {U[13 * n + cell], U[14 * n + cell], U[15 * n + cell]};
        bool ok = isfinite(B[0] + B[1] + B[2] + E[0] + E[1] + E[2]);
        for (int s = 0; s < 2; ++s) {
            double rho = U[(5 * s) * n + cell], p = U[(5 * s + 4) * n + cell];
            double v[3] = {U[(5 * s + 1) * n + cell], U[(5 * s + 2) * n + cell], U[(5 * s + 3) * n + cell]};
            double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            ok = ok && rho > 0.0 && p > 0.0 && v2 < 1.0 && isfinite(rho + p + v2);
            double W = s_rsqrt(1.0 - v2);  // inadmissible states are flagged by ok
            double h = fma(ph.gamma / (ph.gamma - 1.0) * p, s_rcp(rho), 1.0);
            double Z = rho * h * W * W;
            qc[D] += rho * W;
            qc[DB] += mu[s] * rho * W;
            for (int k = 0; k < 3; ++k) {
                qc[SX + k] += Z * v[k];
                qc[SBX + k] += mu[s] * Z * v[k];
            }
            qc[TAU] += Z - p - rho * W;
            qc[TAUB] += mu[s] * (Z - p - rho * W);
            for (int k = 0; k < 3; ++k) w[(5 * s + k) * g.plane + cell] = v[k];
            w[(5 * s + P) * g.plane + cell] = p;
            w[(5 * s + ZZ) * g.plane + cell] = Z;
        }
        if (!ok) { record(status, -1, cell); continue; }
        double ExB[3];
        cross(E, B, ExB);
        for (int k = 0; k < 3; ++k) {
            qc[SX + k] += ExB[k];
            qc[BX + k] = B[k];
            qc[EX + k] = E[k];
        }
        qc[TAU] += 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        for (int k = 0; k < NC; ++k) q[k * g.plane + cell] = qc[k];
    }
}

// Batched runs: Gauss's law within each run (1-D, the run's own boundary map).
__global__ void k_set_prims_batch_sf(Grid g, Phys ph, BatchArgs b, const double *U, double *q, double *w, int *status) {
    using namespace sf;
    const long long n = g.ncell;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        const int run = b.run_of[cell];
        const long long o = b.offset[run];
        const int nx = b.nx[run], i = (int)(cell - o);
        double rho = U[0 * n + cell], v[3] = {U[1 * n + cell], U[2 * n + cell], U[3 * n + cell]}, p = U[4 * n + cell];
        double B[3] = {U[5 * n + cell], U[6 * n + cell], U[7 * n + cell]};
        double E[3] = {U[8 * n + cell], U[9 * n + cell], U[10 * n + cell]};
        double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        bool ok = rho > 0.0 && p > 0.0 && v2 < 1.0 && isfinite(rho + p + v2 + B[0] + B[1] + B[2] + E[0] + E[1] + E[2]);
        if (!ok) { record(status, -1, cell); continue; }
        int il = wrap(i - 1, nx, g.bcx), ir = wrap(i + 1, nx, g.bcx);
        double divE = (U[8 * n + o + ir] - U[8 * n + o + il]) * (2.0 * b.rdx4[run]);
        double W = s_rsqrt(1.0 - v2);  // inadmissible states are flagged by ok
        double h = fma(ph.gamma / (ph.gamma - 1.0) * p, s_rcp(rho), 1.0);
        double Z = rho * h * W * W;
        double ExB[3];
        cross(E, B, ExB);
        double qc[NC];
        qc[D] = rho * W;
        for (int k = 0; k < 3; ++k) {
            qc[SX + k] = Z * v[k] + ExB[k];
            qc[BX + k] = B[k];
            qc[EX + k] = E[k];
        }
        qc[TAU] = Z - p + 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) - rho * W;
        qc[RHOE] = divE;
        qc[PSI] = 0.0;
        qc[PHI] = 0.0;
        for (int k = 0; k < NC; ++k) q[k * g.plane + cell] = qc[k];
        w[VX * g.plane + cell] = v[0];
        w[VY * g.plane + cell] = v[1];
        w[VZ * g.plane + cell] = v[2];
        w[P * g.plane + cell] = p;
        w[LOR * g.plane + cell] = W;
    }
}

cudaError_t launch_set_prims_batch(int model, const Grid &g, const Phys &ph, const BatchArgs &b, const double *prims,
                                   double *q, double *w, int *status, cudaStream_t s) {
    int blocks = grid_for(g.ncell, 256);
    // two fluids have no Gauss's-law initialisation: the per-cell map is the single-grid one
    if (model == 0) k_set_prims_batch_sf<<<blocks, 256, 0, s>>>(g, ph, b, prims, q, w, status);
    else k_set_prims_tf<<<blocks, 256, 0, s>>>(g, ph, prims, q, w, status);
    return cudaGetLastError();
}

cudaError_t launch_set_prims(int model, const Grid &g, const Phys &ph, const double *prims, double *q, double *w,
                             int *status, cudaStream_t s) {
    int blocks = grid_for(g.ncell, 256);
    if (model == 0) k_set_prims_sf<<<blocks, 256, 0, s>>>(g, ph, prims, q, w, status);
    else k_set_prims_tf<<<blocks, 256, 0, s>>>(g, ph, prims, q, w, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- state -> user primitives
// User primitives of one cell from its conserved values q(v) and stored
// primitives w(v) (accessors), written to the dense layout U[var * n + cell].
template <class QF, class WF>
__device__ __forceinline__ void emit_prims_sf(QF q, WF w, double *U, long long n, long long cell) {
    using namespace sf;
    U[0 * n + cell] = q(D) * s_rcp(w(LOR));  // rho = D / W
    U[1 * n + cell] = w(VX);
    U[2 * n + cell] = w(VY);
    U[3 * n + cell] = w(VZ);
    U[4 * n + cell] = w(P);
    for (int k = 0; k < 6; ++k) U[(5 + k) * n + cell] = q(BX + k);
}

template <class QF, class WF>
__device__ __forceinline__ void emit_prims_tf(QF q, WF w, const Phys &ph, double *U, long long n, long long cell) {
    using namespace tf;
    const double Dt = q(D), Db = q(DB);
    const double Ds[2] = {(Db - ph.mu_p * Dt) * ph.inv_dmu, (ph.mu_e * Dt - Db) * ph.inv_dmu};
    for (int s = 0; s < 2; ++s) {
        const double v[3] = {w(5 * s), w(5 * s + 1), w(5 * s + 2)};
        const double om = 1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        U[(5 * s) * n + cell] = Ds[s] * (om * s_rsqrt(om));  // rho_s = D_s / W_s
        for (int k = 0; k < 3; ++k) U[(5 * s + 1 + k) * n + cell] = v[k];
        U[(5 * s + 4) * n + cell] = w(5 * s + P);
    }
    for (int k = 0; k < 6; ++k) U[(10 + k) * n + cell] = q(BX + k);
}

__global__ void k_get_prims_sf(Grid g, const double *q, const double *w, double *U) {
    const long long n = g.ncell;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        emit_prims_sf([&](int v) { return q[v * g.plane + cell]; }, [&](int v) { return w[v * g.plane + cell]; }, U,
                      n, cell);
    }
}

__global__ void k_get_prims_tf(Grid g, Phys ph, const double *q, const double *w, double *U) {
    const long long n = g.ncell;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        emit_prims_tf([&](int v) { return q[v * g.plane + cell]; }, [&](int v) { return w[v * g.plane + cell]; }, ph,
                      U, n, cell);
    }
}

cudaError_t launch_get_prims(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                             double *prims, cudaStream_t s) {
    int blocks = grid_for(g.ncell, 256);
    if (model == 0) k_get_prims_sf<<<blocks, 256, 0, s>>>(g, q, w, prims);
    else k_get_prims_tf<<<blocks, 256, 0, s>>>(g, ph, q, w, prims);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- recovery
// Primitives of q (cold start) into w; with U set, the user primitives of the
// recovered state too (the output of get_prims in one pass, so the recovery
// overlaps the writes when U is host memory).
__global__ void k_recover(int model, Grid g, Phys ph, const double *q, double *w, double *U, int *status) {
    const long long n = g.ncell;
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
         cell += (long long)gridDim.x * blockDim.x) {
        if (model == 0) {
            double qc[sf::NC], wc[sf::NW];
            for (int v = 0; v < sf::NC; ++v) qc[v] = q[v * g.plane + cell];
            // cold start: the recovery brackets the root itself
            int st = sf::recover(qc, -1.0, ph.gamma, wc);
            record(status, st, cell);
            for (int v = 0; v < sf::NW; ++v) w[v * g.plane + cell] = wc[v];
            if (U) emit_prims_sf([&](int v) { return qc[v]; }, [&](int v) { return wc[v]; }, U, n, cell);
        } else {
            double qc[tf::NC], wc[tf::NW], wo[tf::NW];
            for (int v = 0; v < tf::NC; ++v) qc[v] = q[v * g.plane + cell];
            for (int v = 0; v < tf::NW; ++v) wo[v] = -1.0;
            int st = tf::recover(qc, wo, ph, wc);
            record(status, st, cell);
            for (int v = 0; v < tf::NW; ++v) w[v * g.plane + cell] = wc[v];
            if (U) emit_prims_tf([&](int v) { return qc[v]; }, [&](int v) { return wc[v]; }, ph, U, n, cell);
        }
    }
}

cudaError_t launch_recover(int model, const Grid &g, const Phys &ph, const double *q, double *w, int *status,
                           cudaStream_t s, double *prims) {
    k_recover<<<grid_for(g.ncell, 128), 128, 0, s>>>(model, g, ph, q, w, prims, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- layout
__global__ void k_pack(Grid g, int nvar, const double *user, double *dev) {
    long long total = (long long)nvar * g.ncell;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long v = e / g.ncell, c = e - v * g.ncell;
        dev[v * g.plane + c] = user[e];
    }
}
__global__ void k_unpack(Grid g, int nvar, const double *dev, double *user) {
    long long total = (long long)nvar * g.ncell;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long v = e / g.ncell, c = e - v * g.ncell;
        user[e] = dev[v * g.plane + c];
    }
}
cudaError_t launch_pack(const Grid &g, int nvar, const double *user, double *dev, cudaStream_t s) {
    k_pack<<<grid_for((long long)nvar * g.ncell, 256), 256, 0, s>>>(g, nvar, user, dev);
    return cudaGetLastError();
}
cudaError_t launch_unpack(const Grid &g, int nvar, const double *dev, double *user, cudaStream_t s) {
    k_unpack<<<grid_for((long long)nvar * g.ncell, 256), 256, 0, s>>>(g, nvar, dev, user);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- diagnostics
// Two-level deterministic reduction: each of kDiagBlocks blocks reduces a
// strided share of the cells into 8 partials in `scratch`; one block then
// combines the partials in a fixed order.
static constexpr int kDiagBlocks = 304, kDiagThreads = 256;

size_t reduce_scratch_doubles() { return (size_t)kDiagBlocks * 8; }

__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(int model, Grid g, const double *q, const double *w,
                                                               double *scratch) {
    const int NC = model == 0 ? 14 : 18;
    const int iS = 1, iT = 4, iB = model == 0 ? 5 : 10, iR = model == 0 ? 11 : 5;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        acc[0] += q[0 * g.plane + cell];
        acc[1] += q[iT * g.plane + cell];
        acc[2] += q[iS * g.plane + cell];
        acc[3] += q[iB * g.plane + cell];
        acc[4] += q[iR * g.plane + cell];
        for (int s = 0; s < (model == 0 ? 1 : 2); ++s) {
            double vx = w[(5 * s) * g.plane + cell], vy = w[(5 * s + 1) * g.plane + cell], vz = w[(5 * s + 2) * g.plane + cell];
            acc[5] = fmax(acc[5], sqrt(vx * vx + vy * vy + vz * vz));
        }
        double bad = 0.0;
        for (int v = 0; v < NC; ++v) bad += isfinite(q[v * g.plane + cell]) ? 0.0 : 1.0;
        acc[6] += bad;
    }
    __shared__ double red[8][kDiagThreads];
    for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int off = kDiagThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 8; ++k)
                red[k][threadIdx.x] = (k == 5) ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + off])
                                               : red[k][threadIdx.x] + red[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < 8) scratch[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_diag_final(Grid g, double cfl, const double *scratch, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 8; ++k) r[k] = (k == 5) ? fmax(r[k], scratch[b * 8 + k]) : r[k] + scratch[b * 8 + k];
    double vol = g.dx * (g.ny > 1 ? g.dy : 1.0) * (g.nz > 1 ? g.dz : 1.0);
    for (int k = 0; k < 5; ++k) out[k] = r[k] * vol;
    out[5] = r[5];
    out[6] = r[6];
    out[7] = cfl * (g.ny > 1 ? fmin(g.dx, g.dy) : g.dx);
}

cudaError_t launch_diagnostics(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                               double *scratch, double *out, cudaStream_t s) {
    (void)ph;
    k_diag_partial<<<kDiagBlocks, kDiagThreads, 0, s>>>(model, g, q, w, scratch);
    k_diag_final<<<1, 32, 0, s>>>(g, 0.0, scratch, kDiagBlocks, out);
    return cudaGetLastError();
}

} // namespace rmhd
