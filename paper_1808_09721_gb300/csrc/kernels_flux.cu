// kernels_flux.cu -- fused flux-divergence + stage-update kernels.
//
// L(q) = -sum_k (F_{k,+1/2} - F_{k,-1/2}) / dx_k with face fluxes from
// Lax-Friedrichs flux-vector splitting (alpha = 1) and componentwise WENO3
// (Sec. 2.2.2 of Wright & Hawke, arXiv:1808.09721; Jiang-Shu weights with
// eps = 1e-6, power 2).
//
// Formulation used here (algebraically identical to the textbook one). With
// e+- = (f_{i+1} - f_i) +- (q_{i+1} - q_i) at each half point (twice the
// differences of f^+- = (f +- q)/2) and A+- = (4 eps + e+-^2)^2 (a common
// positive multiple of the Jiang-Shu (eps + beta)^2), the face flux is
//   4 F_{i+1/2} = 2 (f_i + f_{i+1}) + w+ (e+_{i-1/2} - e+_{i+1/2}) + w- (e-_{i+1/2} - e-_{i+3/2}),
//   w+ = A+_{i+1/2} / (A+_{i+1/2} + 2 A+_{i-1/2}),  w- = A-_{i+1/2} / (A-_{i+1/2} + 2 A-_{i+3/2}),
// i.e. the central part plus the two nonlinear corrections of the left- and
// right-going reconstructions. Half-point quantities are computed once and
// shared by the two faces that use them; the only division per face and
// sign is one FP64 reciprocal (rcp.approx + one Newton step).
//
// Tiling: one CTA per TX x TY tile, one thread per interior cell. The tile and
// a 2-cell halo of the state are staged in shared memory; boundary conditions
// (outflow = clamp, periodic = wrap) are applied by the halo index map, so no
// ghost cells exist in HBM. Per direction the physical flux of every needed
// cell is computed once into shared memory, then each component is
// reconstructed and differenced. The epilogue fuses the SSP2(222) stage
// update (Table 1) and, after the second pass, the final primitive recovery.
#include "rmhd_internal.h"
#include "physics_sf.cuh"
#include "physics_tf.cuh"

namespace rmhd {

__device__ __forceinline__ int map_index(int i, int n, int bc) {
    if (bc == 1) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

__device__ __forceinline__ void record_status(int *status, int st, long long cell) {
    if (st != 0) {
        atomicCAS(status, 0, st);
        atomicMin(status + 1, (int)cell);
    }
}

// ---- model adaptors ------------------------------------------------------
struct SFModel {
    static constexpr int NC = sf::NC, NW = sf::NW;
    // physical flux of the cell whose state sits at st[v * stride + idx]
    template <class FT>
    static __device__ __forceinline__ void cell_flux(const double *st, int stride, int idx, int dir, const Phys &ph,
                                                     FT f[NC]) {
        double q[NC], w[NW], J[3];
#pragma unroll
        for (int v = 0; v < NC; ++v) q[v] = st[v * stride + idx];
#pragma unroll
        for (int v = 0; v < NW; ++v) w[v] = st[(NC + v) * stride + idx];
        sf::current(q, w, ph.sigma, J);
        FT qf[NC], wf[NW], Jf[3];
#pragma unroll
        for (int v = 0; v < NC; ++v) qf[v] = (FT)q[v];
#pragma unroll
        for (int v = 0; v < NW; ++v) wf[v] = (FT)w[v];
        Jf[0] = (FT)J[0]; Jf[1] = (FT)J[1]; Jf[2] = (FT)J[2];
        sf::flux(qf, wf, Jf, dir, f);
    }
    // source Psi of Eq. (resistive RMHD), nonzero only for E, psi, phi
    static __device__ __forceinline__ void source(const double q[NC], const double w[NW], const Phys &ph, double s[NC]) {
        double J[3];
        sf::current(q, w, ph.sigma, J);
#pragma unroll
        for (int v = 0; v < NC; ++v) s[v] = 0.0;
        s[sf::EX] = -J[0];
        s[sf::EY] = -J[1];
        s[sf::EZ] = -J[2];
        s[sf::PSI] = q[sf::RHOE] - ph.kappa * q[sf::PSI];
        s[sf::PHI] = -ph.kappa * q[sf::PHI];
    }
    static __device__ __forceinline__ int recover(const double q[NC], const double wold[NW], const Phys &ph,
                                                  double w[NW]) {
        return sf::recover(q, wold[sf::P], ph.gamma, w);
    }
};

struct TFModel {
    static constexpr int NC = tf::NC, NW = tf::NW;
    template <class FT>
    static __device__ __forceinline__ void cell_flux(const double *st, int stride, int idx, int dir, const Phys &ph,
                                                     FT f[NC]) {
        FT qf[NC], wf[NW];
#pragma unroll
        for (int v = 0; v < NC; ++v) qf[v] = (FT)st[v * stride + idx];
#pragma unroll
        for (int v = 0; v < NW; ++v) wf[v] = (FT)st[(NC + v) * stride + idx];
        tf::flux(qf, wf, (FT)ph.mu_e, (FT)ph.mu_p, (FT)ph.inv_dmu, dir, f);
    }
    static __device__ __forceinline__ void source(const double q[NC], const double w[NW], const Phys &ph, double s[NC]) {
        tf::source(q, w, ph, s);
    }
    static __device__ __forceinline__ int recover(const double q[NC], const double wold[NW], const Phys &ph,
                                                  double w[NW]) {
        return tf::recover(q, wold, ph, w);
    }
};

// ---- the fused flux kernel -----------------------------------------------
template <class M, int TX, int TY, class FT, int MODE>
__global__ void __launch_bounds__(TX *TY, 1) k_flux(Grid g, Phys ph, FluxArgs a) {
    constexpr int NC = M::NC, NW = M::NW, NV = NC + NW;
    constexpr bool TWO_D = TY > 1;
    constexpr int SW = TX + 4, SH = TWO_D ? TY + 4 : 1, SN = SW * SH;
    constexpr int NT = TX * TY;
    constexpr int OY = TWO_D ? 2 : 0;  // SMEM row of the first interior row

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *st = reinterpret_cast<double *>(smem_raw);            // [NV][SH][SW]
    FT *fl = reinterpret_cast<FT *>(st + NV * SN);                 // [NC][SH][SW]
    FT *hp = fl + NC * SN;                                         // [4][SH][SW]: e+, e-, A+, A-
    FT *fc = hp + 4 * SN;                                          // [SH][SW]: 4 F at the face right of the cell

    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;

    // 1. stage the tile + halo (boundary conditions by index map)
    for (int e = tid; e < NV * SN; e += NT) {
        int v = e / SN, r = e - v * SN;
        int sy = r / SW, sx = r - sy * SW;
        int gi = map_index(i0 + sx - 2, g.nx, g.bcx);
        int gj = TWO_D ? map_index(j0 + sy - 2, g.ny, g.bcy) : 0;
        const double *src = v < NC ? a.q + (long long)v * g.plane : a.w + (long long)(v - NC) * g.plane;
        st[e] = src[(long long)gj * g.nx + gi];
    }
    __syncthreads();

    const int tx = tid % TX, ty = tid / TX;
    const int ox = tx + 2, oy = ty + OY;  // owner cell in SMEM coordinates
    FT L[NC];
#pragma unroll
    for (int v = 0; v < NC; ++v) L[v] = FT(0);

    const FT eps4 = FT(4e-6);
#pragma unroll 1
    for (int dir = 0; dir < (TWO_D ? 2 : 1); ++dir) {
        const int sstep = dir == 0 ? 1 : SW;  // SMEM offset of the next cell along dir
        const FT inv4h = FT(0.25 / (dir == 0 ? g.dx : g.dy));
        // 2a. physical flux of every cell the reconstruction needs
        const int ncx = dir == 0 ? SW : TX, ncy = dir == 0 ? TY : SH;
        const int cx0 = dir == 0 ? 0 : 2, cy0 = dir == 0 ? OY : 0;
        for (int e = tid; e < ncx * ncy; e += NT) {
            int cy = e / ncx, cx = e - cy * ncx;
            int idx = (cy0 + cy) * SW + cx0 + cx;
            FT f[NC];
            M::template cell_flux<FT>(st, SN, idx, dir, ph, f);
#pragma unroll
            for (int v = 0; v < NC; ++v) fl[v * SN + idx] = f[v];
        }
        __syncthreads();
        // half points between cell c and c + sstep: along dir, from the first
        // halo cell to the last-but-one
        const int nhx = dir == 0 ? SW - 1 : TX, nhy = dir == 0 ? TY : SH - 1;
        const int hx0 = dir == 0 ? 0 : 2, hy0 = dir == 0 ? OY : 0;
        // faces right of cells 1 .. T+1 (SMEM coordinate along dir)
        const int nfx = dir == 0 ? TX + 1 : TX, nfy = dir == 0 ? TY : TY + 1;
        const int fx0 = dir == 0 ? 1 : 2, fy0 = dir == 0 ? OY : 1;
#pragma unroll 1
        for (int c = 0; c < NC; ++c) {
            const FT *fv = fl + c * SN;
            const double *qv = st + c * SN;
            for (int e = tid; e < nhx * nhy; e += NT) {
                int hy = e / nhx, hx = e - hy * nhx;
                int idx = (hy0 + hy) * SW + hx0 + hx;
                FT df = fv[idx + sstep] - fv[idx];
                FT dq = FT(qv[idx + sstep] - qv[idx]);
                FT ep = df + dq, em = df - dq;
                FT ap = eps4 + ep * ep, am = eps4 + em * em;
                hp[idx] = ep;
                hp[SN + idx] = em;
                hp[2 * SN + idx] = ap * ap;
                hp[3 * SN + idx] = am * am;
            }
            __syncthreads();
            for (int e = tid; e < nfx * nfy; e += NT) {
                int fy = e / nfx, fx = e - fy * nfx;
                int idx = (fy0 + fy) * SW + fx0 + fx;
                int il = idx - sstep, ir = idx + sstep;
                FT Ap = hp[2 * SN + idx], Am = hp[3 * SN + idx];
                FT wp = Ap * s_rcp1(Ap + FT(2) * hp[2 * SN + il]);
                FT wm = Am * s_rcp1(Am + FT(2) * hp[3 * SN + ir]);
                FT Xp = hp[il] - hp[idx];
                FT Xm = hp[SN + idx] - hp[SN + ir];
                fc[idx] = s_fma(FT(2), fv[idx] + fv[ir], s_fma(wp, Xp, wm * Xm));
            }
            __syncthreads();
            L[c] = s_fma(fc[oy * SW + ox - sstep] - fc[oy * SW + ox], inv4h, L[c]);
        }
        __syncthreads();
    }

    // 3. epilogue for the owner cell
    const int gi = i0 + tx, gj = j0 + ty;
    if (gi >= g.nx || gj >= g.ny) return;
    const long long cell = (long long)gj * g.nx + gi;
    const int oidx = oy * SW + ox;
    double q[NC], w[NW], s[NC];
#pragma unroll
    for (int v = 0; v < NC; ++v) q[v] = st[v * SN + oidx];
#pragma unroll
    for (int v = 0; v < NW; ++v) w[v] = st[(NC + v) * SN + oidx];
    M::source(q, w, ph, s);
    const double dt = a.dt, hdt = 0.5 * a.dt;
    if (MODE == 1) {
        const double cs = a.c_src * a.dt;
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            double b = a.base[v * g.plane + cell];
            double Lv = (double)L[v];
            a.out1[v * g.plane + cell] = fma(cs, s[v], fma(dt, Lv, b));
            a.out2[v * g.plane + cell] = fma(hdt, Lv + s[v], b);
        }
    } else {
        double qn[NC], wn[NW];
#pragma unroll
        for (int v = 0; v < NC; ++v) {
            qn[v] = fma(hdt, (double)L[v] + s[v], a.base[v * g.plane + cell]);
            a.out1[v * g.plane + cell] = qn[v];
        }
        int stc = M::recover(qn, w, ph, wn);
        record_status(a.status, stc, cell);
#pragma unroll
        for (int v = 0; v < NW; ++v) a.out2[v * g.plane + cell] = wn[v];
    }
}

template <class M, int TX, int TY, class FT>
static size_t flux_smem() {
    constexpr int NC = M::NC, NW = M::NW;
    constexpr int SW = TX + 4, SH = TY > 1 ? TY + 4 : 1, SN = SW * SH;
    return (size_t)(NC + NW) * SN * sizeof(double) + (size_t)(NC + 5) * SN * sizeof(FT);
}

template <class M, int TX, int TY, class FT, int MODE>
static cudaError_t launch_flux_t(const Grid &g, const Phys &ph, const FluxArgs &a, cudaStream_t s) {
    size_t smem = flux_smem<M, TX, TY, FT>();
    static bool configured = false;  // attribute is per device function; set once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_flux<M, TX, TY, FT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((g.nx + TX - 1) / TX, TY > 1 ? (g.ny + TY - 1) / TY : g.ny);
    k_flux<M, TX, TY, FT, MODE><<<grid, TX * TY, smem, s>>>(g, ph, a);
    return cudaGetLastError();
}

template <class M, class FT, int MODE>
static cudaError_t launch_flux_m(const Grid &g, const Phys &ph, const FluxArgs &a, cudaStream_t s) {
    if (g.ny == 1) return launch_flux_t<M, 128, 1, FT, MODE>(g, ph, a, s);
    return launch_flux_t<M, 32, 8, FT, MODE>(g, ph, a, s);
}

cudaError_t launch_flux(int model, int precision, int mode, const Grid &g, const Phys &ph, const FluxArgs &a,
                        cudaStream_t s) {
    if (model == 0) {
        if (precision == 0)
            return mode == 1 ? launch_flux_m<SFModel, double, 1>(g, ph, a, s) : launch_flux_m<SFModel, double, 2>(g, ph, a, s);
        return mode == 1 ? launch_flux_m<SFModel, float, 1>(g, ph, a, s) : launch_flux_m<SFModel, float, 2>(g, ph, a, s);
    }
    if (precision == 0)
        return mode == 1 ? launch_flux_m<TFModel, double, 1>(g, ph, a, s) : launch_flux_m<TFModel, double, 2>(g, ph, a, s);
    return mode == 1 ? launch_flux_m<TFModel, float, 1>(g, ph, a, s) : launch_flux_m<TFModel, float, 2>(g, ph, a, s);
}

} // namespace rmhd
