// kernels_adjoint.cu -- discrete adjoint of the SSP2(222) IMEX step (single
// fluid, FP64) of Wright & Hawke, arXiv:1808.09721 (Sec. 2.2.1, Table 1;
// Sec. 2.2.2 fluxes; Sec. 2.1.1 model).
//
// Reverse of one SSP2(222) step, with lambda the adjoint of q^{n+1}, (q_i, w_i)
// the stored stage states and g = 1 - 1/sqrt(2):
//   lambda_q2 = (dL/dq)^T (dt/2 lambda) + (dPsi/dq)^T (dt/2 lambda)    at q2
//   lambda_r2 = (I - g dt dPsi/dq)^{-T} lambda_q2                       at q2
//   lambda_q1 = (dL/dq)^T (dt lambda_r2 + dt/2 lambda)
//             + (dPsi/dq)^T ((1 - 2g) dt lambda_r2 + dt/2 lambda)       at q1
//   lambda^n  = (I - g dt dPsi/dq)^{-T} lambda_q1 + lambda_r2 + lambda  at q1
// SSP3(332) (Table 2: R = q^n + dt L1 + (1 - 2g) dt Psi1, R3 = q^n + dt/4 (L1 +
// L2) + (1/2 - g) dt Psi1, q^{n+1} = q^n + dt/6 (L1 + Psi1 + L2 + Psi2) + 2 dt/3
// (L3 + Psi3)) reverses the same way, stage 3 first:
//   lambda_R3 = S3^T [(dL/dq)^T + (dPsi/dq)^T] (2 dt/3 lambda)              at q3
//   lambda_R  = S2^T [(dL/dq)^T (dt/6 lambda + dt/4 lambda_R3) + (dPsi/dq)^T (dt/6 lambda)]   at q2
//   lambda^n  = S1^T [(dL/dq)^T (dt/6 lambda + dt/4 lambda_R3 + dt lambda_R)
//             + (dPsi/dq)^T (dt/6 lambda + (1/2 - g) dt lambda_R3 + (1 - 2g) dt lambda_R)]
//             + lambda_R + lambda_R3 + lambda                               at q1
// with S_i^T = (I - g dt dPsi/dq)^{-T} at q_i.
// The stage solves are differentiated by the implicit-function theorem, the
// primitive recovery inside every map likewise (adjoint_sf.cuh). The flux
// divergence is transposed face by face: each face's WENO3/LF value depends on
// four stencil cells (mapped through the boundary conditions); its reverse
// scatters into their flux- and state-adjoints with FP64 atomics.
//
// Intermediates live in global memory (one plane per variable): the sweep is
// bound by FP64 arithmetic, not by HBM, so simple per-cell and per-face
// kernels are used instead of a fused tile.
//
// Two fluids (MODEL = 1): the same reverse sweep with the 18 conserved
// variables; the stiff unknowns of a stage are (Sbar, taubar, E), so the
// stage adjoint solves a 7 x 7 transposed system (adjoint_tf.cuh has the cell
// maps' vector-Jacobian products).
#include "rmhd_internal.h"
#include "adjoint_sf.cuh"
#include "adjoint_tf.cuh"

namespace rmhd {

namespace {

__device__ __forceinline__ int amap(int i, int n, int bc) {
    if (bc == 1) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// A weighted sum of up to three adjoint fields: sum a[k] p[k][i] (null p[k] skipped).
struct Lin {
    const double *p[3];
    double a[3];
    __device__ __forceinline__ double at(long long i) const {
        double s = 0.0;
        for (int k = 0; k < 3; ++k)
            if (p[k]) s += a[k] * p[k][i];
        return s;
    }
};

// Per-model sizes and cell maps of the reverse sweep.
template <int MODEL> struct AdjModel;
template <> struct AdjModel<0> {
    static constexpr int NC = sf::NC, NW = sf::NW, NS = 5, NX = 3, NP = 11;
    // source entries (E, psi, phi) in the order cell_vjp takes their adjoints
    static __device__ __forceinline__ int src(int k) { return k < 3 ? sf::EX + k : (k == 3 ? sf::PSI : sf::PHI); }
    static __device__ __forceinline__ void flux(const double *qc, const double *wc, const Phys &ph, int dir, double *f) {
        double J[3];
        sf::current(qc, wc, ph.sigma, J);
        sf::flux(qc, wc, J, dir, f);
    }
    static __device__ __forceinline__ void vjp(const double *qc, const double *wc, const Phys &ph, int ndir,
                                               const double fb[3][NC], const double *sb, double *qb, double *sigb) {
        sf::cell_vjp(qc, wc[sf::P], ph.gamma, ph.sigma, ph.kappa, ndir, fb, sb, qb, sigb);
    }
};
template <> struct AdjModel<1> {
    static constexpr int NC = tf::NC, NW = tf::NW, NS = 9, NX = 7, NP = 16;
    // source entries (Sbar, taubar, E, psi, phi); the first NX are the stage unknowns
    static __device__ __forceinline__ int src(int k) {
        return k < 4 ? tf::SBX + k : (k < 7 ? tf::EX + k - 4 : (k == 7 ? tf::PSI : tf::PHI));
    }
    static __device__ __forceinline__ void flux(const double *qc, const double *wc, const Phys &ph, int dir, double *f) {
        tf::flux<double>(qc, wc, ph.mu_e, ph.mu_p, ph.inv_dmu, dir, f);
    }
    static __device__ __forceinline__ void vjp(const double *qc, const double *wc, const Phys &ph, int ndir,
                                               const double fb[3][NC], const double *sb, double *qb, double *sigb) {
        tf::cell_vjp(qc, wc, ph, ndir, fb, sb, qb, sigb);
    }
};

// Physical fluxes f_x, f_y, f_z (N_c each; y, z where the grid has them) of
// every cell of a stage state.
template <int MODEL>
__global__ void k_cellflux(Grid g, Phys ph, const double *q, const double *w, double *fx, double *fy, double *fz) {
    using Mo = AdjModel<MODEL>;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double qc[Mo::NC], wc[Mo::NW], f[Mo::NC];
        for (int v = 0; v < Mo::NC; ++v) qc[v] = q[v * g.plane + c];
        for (int v = 0; v < Mo::NW; ++v) wc[v] = w[v * g.plane + c];
        Mo::flux(qc, wc, ph, 0, f);
        for (int v = 0; v < Mo::NC; ++v) fx[v * g.plane + c] = f[v];
        if (g.ny > 1) {
            Mo::flux(qc, wc, ph, 1, f);
            for (int v = 0; v < Mo::NC; ++v) fy[v * g.plane + c] = f[v];
        }
        if (g.nz > 1) {
            Mo::flux(qc, wc, ph, 2, f);
            for (int v = 0; v < Mo::NC; ++v) fz[v * g.plane + c] = f[v];
        }
    }
}

// Reverse of the face values along `dir`. One thread per (face, component):
// faces k = -1 .. n-1 along dir (the face after cell k) for every line.
// Consecutive threads take neighbouring faces along x (dir 0) or neighbouring
// lines (dir 1), so a warp's loads and atomics fall on consecutive cells of
// one variable plane. lamL_ = the adjoint of L (a weighted sum of adjoint fields).
__global__ void k_face_adj(Grid g, int dir, int ncomp, const double *q, const double *f, Lin lamL_, double *fbar,
                           double *qbar) {
    const int nz = g.nz > 1 ? g.nz : 1;
    const long long nxy = (long long)g.nx * g.ny;
    // cells along dir, lines across it
    const int n = dir == 0 ? g.nx : (dir == 1 ? g.ny : nz);
    const long long m = dir == 0 ? (long long)g.ny * nz : (dir == 1 ? (long long)g.nx * nz : nxy);
    const int bc = dir == 0 ? g.bcx : (dir == 1 ? g.bcy : g.bcz);
    const double h4 = dir == 0 ? g.rdx4 : (dir == 1 ? g.rdy4 : g.rdz4);
    const long long nf = (long long)(n + 1) * m * ncomp;
    const double eps4 = 4e-6;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nf; t += (long long)gridDim.x * blockDim.x) {
        int c, k;        // component, face after cell k
        long long line;  // dir 0: (z, y) row; dir 1: (z, x) column; dir 2: (y, x) pillar
        if (dir == 0) {
            k = (int)(t % (n + 1)) - 1;
            const long long r = t / (n + 1);
            line = r % m;
            c = (int)(r / m);
        } else {
            line = t % m;
            const long long r = t / m;
            k = (int)(r % (n + 1)) - 1;
            c = (int)(r / (n + 1));
        }
        auto cell = [&](int i) -> long long {
            const long long im = amap(i, n, bc);
            if (dir == 0) return line * g.nx + im;
            if (dir == 1) return (line / g.nx) * nxy + im * g.nx + line % g.nx;
            return im * nxy + line;
        };
        auto lamL = [&](long long cc) -> double { return lamL_.at(c * g.plane + cc); };
        // 4F at this face enters L of cell k (- 1/(4h)) and of cell k+1 (+ 1/(4h)), real cells only
        double Fb = 0.0;
        if (k >= 0) Fb -= h4 * lamL(cell(k));
        if (k + 1 < n) Fb += h4 * lamL(cell(k + 1));
        if (Fb == 0.0) continue;
        long long cs[4];
        double fs[4], qs[4];
        for (int s = 0; s < 4; ++s) {
            cs[s] = cell(k - 1 + s);
            fs[s] = f[c * g.plane + cs[s]];
            qs[s] = q[c * g.plane + cs[s]];
        }
        // half points j = 0, 1, 2 between stencil cells (j, j+1)
        double ep[3], em[3], Ap[3], Am[3], sp[3], sm[3];
        for (int j = 0; j < 3; ++j) {
            double df = fs[j + 1] - fs[j], dq = qs[j + 1] - qs[j];
            ep[j] = df + dq;
            em[j] = df - dq;
            sp[j] = eps4 + ep[j] * ep[j];
            sm[j] = eps4 + em[j] * em[j];
            Ap[j] = sp[j] * sp[j];
            Am[j] = sm[j] * sm[j];
        }
        const double denp = Ap[1] + 2.0 * Ap[0], denm = Am[1] + 2.0 * Am[2];
        const double rdp = s_rcp(denp), rdm = s_rcp(denm);
        const double wp = Ap[1] * rdp, wm = Am[1] * rdm;
        const double Xp = ep[0] - ep[1], Xm = em[1] - em[2];
        // reverse
        double fb[4] = {0, 2.0 * Fb, 2.0 * Fb, 0}, qb[4] = {0, 0, 0, 0};
        double epb[3] = {0, 0, 0}, emb[3] = {0, 0, 0}, Apb[3] = {0, 0, 0}, Amb[3] = {0, 0, 0};
        const double wpb = Fb * Xp, Xpb = Fb * wp, wmb = Fb * Xm, Xmb = Fb * wm;
        epb[0] += Xpb;
        epb[1] -= Xpb;
        emb[1] += Xmb;
        emb[2] -= Xmb;
        Apb[1] += wpb * 2.0 * Ap[0] * rdp * rdp;
        Apb[0] -= wpb * 2.0 * Ap[1] * rdp * rdp;
        Amb[1] += wmb * 2.0 * Am[2] * rdm * rdm;
        Amb[2] -= wmb * 2.0 * Am[1] * rdm * rdm;
        for (int j = 0; j < 3; ++j) {
            epb[j] += Apb[j] * 4.0 * ep[j] * sp[j];
            emb[j] += Amb[j] * 4.0 * em[j] * sm[j];
            const double dfb = epb[j] + emb[j], dqb = epb[j] - emb[j];
            fb[j + 1] += dfb;
            fb[j] -= dfb;
            qb[j + 1] += dqb;
            qb[j] -= dqb;
        }
        for (int s = 0; s < 4; ++s) {
            atomicAdd(&fbar[c * g.plane + cs[s]], fb[s]);
            atomicAdd(&qbar[c * g.plane + cs[s]], qb[s]);
        }
    }
}

// Per cell: lambda_q = qbar (direct, from the splitting) + cell_vjp(fbar_x, fbar_y, sbar),
// sbar = the adjoint of Psi (a weighted sum of adjoint fields) at the source
// components. Adds the sigma adjoint into sig[cell].
template <int MODEL>
__global__ void k_cell_adj(Grid g, Phys ph, const double *q, const double *w, const double *fbx, const double *fby,
                           const double *fbz, const double *qbd, Lin psib, double *lamq, double *sig) {
    using Mo = AdjModel<MODEL>;
    const int ndir = g.nz > 1 ? 3 : (g.ny > 1 ? 2 : 1);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double qc[Mo::NC], wc[Mo::NW], qb[Mo::NC], fb[3][Mo::NC], sb[Mo::NS];
        for (int v = 0; v < Mo::NC; ++v) {
            qc[v] = q[v * g.plane + c];
            qb[v] = qbd[v * g.plane + c];
            fb[0][v] = fbx[v * g.plane + c];
            fb[1][v] = ndir > 1 ? fby[v * g.plane + c] : 0.0;
            fb[2][v] = ndir > 2 ? fbz[v * g.plane + c] : 0.0;
        }
        for (int v = 0; v < Mo::NW; ++v) wc[v] = w[v * g.plane + c];
        for (int k = 0; k < Mo::NS; ++k) sb[k] = psib.at(Mo::src(k) * g.plane + c);
        double sigb = 0.0;
        Mo::vjp(qc, wc, ph, ndir, fb, sb, qb, &sigb);
        for (int v = 0; v < Mo::NC; ++v) lamq[v * g.plane + c] = qb[v];
        sig[c] += sigb;
    }
}

// Implicit-stage adjoint at the stage state q: mu = (I - adt dPsi/dq)^{-T} lambda.
// Psi has nonzero rows only for the stiff unknowns x (one fluid: E; two
// fluids: Sbar, taubar, E) and psi, phi: the NX x NX block of x is solved
// exactly (rows of dPsi_x/dx by NX reverse products, then Gaussian
// elimination with partial pivoting of the transposed system), psi and phi
// scale by 1/(1 + adt kappa), and the other components are
// mu_n = lambda_n + adt [(dPsi/dq)^T mu_src]_n. out = mu + the fields of add
// (weights 1; null entries skipped).
template <int MODEL>
__global__ void k_stage_adj(Grid g, Phys ph, double adt, const double *q, const double *w, const double *lam,
                            Lin add, double *out, double *sig) {
    using Mo = AdjModel<MODEL>;
    constexpr int NC = Mo::NC, NX = Mo::NX, NS = Mo::NS;
    const double nofb[3][NC] = {};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double qc[NC], wc[Mo::NW], la[NC];
        for (int v = 0; v < NC; ++v) {
            qc[v] = q[v * g.plane + c];
            la[v] = lam[v * g.plane + c];
        }
        for (int v = 0; v < Mo::NW; ++v) wc[v] = w[v * g.plane + c];
        // M = (I - adt A)^T with A[i][j] = dPsi_{x_i}/dx_j; M[j][i] = delta_ji - adt A[i][j]
        double M[NX][NX + 1];
        for (int i = 0; i < NX; ++i) {
            double sb[NS] = {}, qb[NC] = {}, sgd = 0.0;
            sb[i] = 1.0;
            Mo::vjp(qc, wc, ph, 0, nofb, sb, qb, &sgd);
            for (int j = 0; j < NX; ++j) M[j][i] = (i == j ? 1.0 : 0.0) - adt * qb[Mo::src(j)];
        }
        for (int j = 0; j < NX; ++j) M[j][NX] = la[Mo::src(j)];
        // Gaussian elimination with partial pivoting (row swaps by compare and
        // select, so that every index is a compile-time constant), then back
        // substitution
#pragma unroll
        for (int k = 0; k < NX; ++k) {
#pragma unroll
            for (int r = k + 1; r < NX; ++r)
                if (fabs(M[r][k]) > fabs(M[k][k]))
#pragma unroll
                    for (int j = k; j <= NX; ++j) { const double t = M[k][j]; M[k][j] = M[r][j]; M[r][j] = t; }
            const double ip = 1.0 / M[k][k];
            for (int r = k + 1; r < NX; ++r) {
                const double f = M[r][k] * ip;
                for (int j = k; j <= NX; ++j) M[r][j] -= f * M[k][j];
            }
        }
        double mu[NS];
        for (int k = NX - 1; k >= 0; --k) {
            double t = M[k][NX];
            for (int j = k + 1; j < NX; ++j) t -= M[k][j] * mu[j];
            mu[k] = t / M[k][k];
        }
        const double ck = 1.0 / (1.0 + adt * ph.kappa);
        mu[NX] = la[Mo::src(NX)] * ck;          // psi
        mu[NX + 1] = la[Mo::src(NX + 1)] * ck;  // phi
        double qb[NC] = {}, sgb = 0.0;
        Mo::vjp(qc, wc, ph, 0, nofb, mu, qb, &sgb);
        double o[NC];
        for (int v = 0; v < NC; ++v) o[v] = la[v] + adt * qb[v];
        for (int k = 0; k < NS; ++k) o[Mo::src(k)] = mu[k];
        for (int v = 0; v < NC; ++v) out[v * g.plane + c] = o[v] + add.at(v * g.plane + c);
        sig[c] += adt * sgb;
    }
}

// Adjoint of the initial map (user primitives -> conserved state, Gauss's
// law varrho = div E by central differences with the boundary map; psi = phi
// = 0 are constants). pbar: 11 planes, E planes accumulated atomically.
__global__ void k_prims_adj(Grid g, Phys ph, const double *q, const double *w, const double *lam, double *pbar) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double qb[sf::NC], prim[11], pb[11];
        for (int v = 0; v < sf::NC; ++v) qb[v] = lam[v * g.plane + c];
        const double W = w[sf::LOR * g.plane + c];
        prim[0] = q[sf::D * g.plane + c] / W;
        for (int i = 0; i < 3; ++i) prim[1 + i] = w[(sf::VX + i) * g.plane + c];
        prim[4] = w[sf::P * g.plane + c];
        for (int i = 0; i < 6; ++i) prim[5 + i] = q[(sf::BX + i) * g.plane + c];
        sf::p2c_vjp(prim, ph.gamma, qb, pb);
        for (int k = 0; k < 11; ++k) atomicAdd(&pbar[k * g.plane + c], pb[k]);
        // varrho_c = (E_x[i+1] - E_x[i-1]) / (2 dx) + (E_y[j+1] - E_y[j-1]) / (2 dy)
        //          + (E_z[k+1] - E_z[k-1]) / (2 dz)
        const double lr = qb[sf::RHOE];
        const long long nxy = (long long)g.nx * g.ny;
        const int kz = (int)(c / nxy);
        const long long rem = c - kz * nxy, pz = kz * nxy;
        const int j = (int)(rem / g.nx), i = (int)(rem - (long long)j * g.nx);
        const double hx = lr / (2.0 * g.dx);
        atomicAdd(&pbar[8 * g.plane + pz + (long long)j * g.nx + amap(i + 1, g.nx, g.bcx)], hx);
        atomicAdd(&pbar[8 * g.plane + pz + (long long)j * g.nx + amap(i - 1, g.nx, g.bcx)], -hx);
        if (g.ny > 1) {
            const double hy = lr / (2.0 * g.dy);
            atomicAdd(&pbar[9 * g.plane + pz + (long long)amap(j + 1, g.ny, g.bcy) * g.nx + i], hy);
            atomicAdd(&pbar[9 * g.plane + pz + (long long)amap(j - 1, g.ny, g.bcy) * g.nx + i], -hy);
        }
        if (g.nz > 1) {
            const double hz = lr / (2.0 * g.dz);
            atomicAdd(&pbar[10 * g.plane + (long long)amap(kz + 1, g.nz, g.bcz) * nxy + rem], hz);
            atomicAdd(&pbar[10 * g.plane + (long long)amap(kz - 1, g.nz, g.bcz) * nxy + rem], -hz);
        }
    }
}

// Two fluids: adjoint of the initial map (user primitives -> conserved state,
// Eq. twoFluid cons; psi = phi = 0 are constants, no Gauss's law: the charge
// Dbar follows from the species densities). pbar: 16 planes.
__global__ void k_prims_adj_tf(Grid g, Phys ph, const double *q, const double *w, const double *lam, double *pbar) {
    const tf::Split sp(ph.mu_e, ph.mu_p, ph.inv_dmu);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double qb[tf::NC], prim[16], pb[16];
        for (int v = 0; v < tf::NC; ++v) qb[v] = lam[v * g.plane + c];
        const double D = q[tf::D * g.plane + c], Db = q[tf::DB * g.plane + c];
        const double Ds[2] = {sp.ce_bar * Db + sp.ce_tot * D, sp.cp_bar * Db + sp.cp_tot * D};
        for (int s = 0; s < 2; ++s) {
            double v[3];
            for (int i = 0; i < 3; ++i) v[i] = w[(5 * s + tf::VX + i) * g.plane + c];
            const double W = 1.0 / sqrt(1.0 - sf::dot3(v, v));
            prim[5 * s] = Ds[s] / W;
            for (int i = 0; i < 3; ++i) prim[5 * s + 1 + i] = v[i];
            prim[5 * s + 4] = w[(5 * s + tf::P) * g.plane + c];
        }
        for (int i = 0; i < 6; ++i) prim[10 + i] = q[(tf::BX + i) * g.plane + c];
        tf::p2c_vjp(prim, ph, qb, pb);
        for (int k = 0; k < 16; ++k) pbar[k * g.plane + c] = pb[k];
    }
}

// Deterministic single-block sum of a plane.
__global__ void k_sum(const double *x, long long n, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

int blocks_for(long long n, int t) {
    long long b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : (b > (1 << 20) ? (1 << 20) : b));
}

} // namespace

// Reverse of one stage at the stored stage state (q, w): lambda_q from the
// transposed flux divergence (adjoint of L: lamL) and the source VJP
// (adjoint of Psi: psib), then out = S^T lambda_q + the fields of add.
template <int MODEL>
static cudaError_t reverse_stage(const Grid &g, const Phys &ph, double adt, const double *q, const double *w,
                                 Lin lamL, Lin psib, Lin add, double *out, double *const *f, double *const *fb,
                                 double *qbd, double *lq, double *sig, cudaStream_t s) {
    constexpr int NC = AdjModel<MODEL>::NC;
    const size_t pb = (size_t)g.plane * NC * sizeof(double);
    const int T = 256;
    const int cb = blocks_for(g.ncell, T);
    const int ndir = g.nz > 1 ? 3 : (g.ny > 1 ? 2 : 1);
    const long long nz = g.nz > 1 ? g.nz : 1;
    for (int d = 0; d < ndir; ++d) cudaMemsetAsync(fb[d], 0, pb, s);
    cudaMemsetAsync(qbd, 0, pb, s);
    k_cellflux<MODEL><<<cb, T, 0, s>>>(g, ph, q, w, f[0], f[1], f[2]);
    for (int d = 0; d < ndir; ++d) {
        // (cells along d + 1 faces) x lines across d x components
        const long long n = d == 0 ? g.nx : (d == 1 ? g.ny : nz);
        const long long lines = g.ncell / n;
        const long long nf = (n + 1) * lines * NC;
        k_face_adj<<<blocks_for(nf, T), T, 0, s>>>(g, d, NC, q, f[d], lamL, fb[d], qbd);
    }
    k_cell_adj<MODEL><<<cb, T, 0, s>>>(g, ph, q, w, fb[0], fb[1], fb[2], qbd, psib, lq, sig);
    k_stage_adj<MODEL><<<cb, T, 0, s>>>(g, ph, adt, q, w, lq, add, out, sig);
    return cudaGetLastError();
}

// One reverse step; see the file comment. lam (in) -> out (lambda^n); Sq/Sw the
// stage states (2 for SSP2(222), 3 for SSP3(332)); scratch planes: f[3] cell
// fluxes and fb[3] their adjoints (x, y, z; those the grid has), qbd, lq, lr2,
// lr3 (SSP3 only); sig the per-cell sigma adjoint (accumulated).
template <int MODEL>
static cudaError_t adjoint_step_t(const Grid &g, const Phys &ph, int scheme, double dt, const double *lam, double *out,
                                  const double *const *Sq, const double *const *Sw, double *const *f,
                                  double *const *fb, double *qbd, double *lq, double *lr2, double *lr3,
                                  double *sig, cudaStream_t s) {
    const double gam = 1.0 - 0.70710678118654752440;
    const double adt = gam * dt;
    const Lin none{{nullptr, nullptr, nullptr}, {0.0, 0.0, 0.0}};
    cudaError_t e;
    if (scheme == 0) {
        // stage 2: L2 and Psi2 enter q^{n+1} with dt/2
        const Lin l2{{lam, nullptr, nullptr}, {0.5 * dt, 0.0, 0.0}};
        e = reverse_stage<MODEL>(g, ph, adt, Sq[1], Sw[1], l2, l2, none, lr2, f, fb, qbd, lq, sig, s);
        if (e != cudaSuccess) return e;
        // stage 1: L1 enters r2 (dt) and q^{n+1} (dt/2); Psi1 with (1 - 2g) dt and dt/2
        const Lin l1{{lr2, lam, nullptr}, {dt, 0.5 * dt, 0.0}};
        const Lin p1{{lr2, lam, nullptr}, {(1.0 - 2.0 * gam) * dt, 0.5 * dt, 0.0}};
        const Lin a1{{lr2, lam, nullptr}, {1.0, 1.0, 0.0}};
        return reverse_stage<MODEL>(g, ph, adt, Sq[0], Sw[0], l1, p1, a1, out, f, fb, qbd, lq, sig, s);
    }
    // SSP3(332), stage 3: L3 and Psi3 enter q^{n+1} with 2 dt/3
    const Lin l3{{lam, nullptr, nullptr}, {2.0 * dt / 3.0, 0.0, 0.0}};
    e = reverse_stage<MODEL>(g, ph, adt, Sq[2], Sw[2], l3, l3, none, lr3, f, fb, qbd, lq, sig, s);
    if (e != cudaSuccess) return e;
    // stage 2: L2 enters q^{n+1} (dt/6) and R3 (dt/4); Psi2 only q^{n+1} (dt/6)
    const Lin l2{{lam, lr3, nullptr}, {dt / 6.0, 0.25 * dt, 0.0}};
    const Lin p2{{lam, nullptr, nullptr}, {dt / 6.0, 0.0, 0.0}};
    e = reverse_stage<MODEL>(g, ph, adt, Sq[1], Sw[1], l2, p2, none, lr2, f, fb, qbd, lq, sig, s);
    if (e != cudaSuccess) return e;
    // stage 1: L1 enters q^{n+1} (dt/6), R3 (dt/4) and R (dt); Psi1 with dt/6,
    // (1/2 - g) dt and (1 - 2g) dt; q^n enters all three with weight 1
    const Lin l1{{lam, lr3, lr2}, {dt / 6.0, 0.25 * dt, dt}};
    const Lin p1{{lam, lr3, lr2}, {dt / 6.0, (0.5 - gam) * dt, (1.0 - 2.0 * gam) * dt}};
    const Lin a1{{lam, lr3, lr2}, {1.0, 1.0, 1.0}};
    return reverse_stage<MODEL>(g, ph, adt, Sq[0], Sw[0], l1, p1, a1, out, f, fb, qbd, lq, sig, s);
}

cudaError_t launch_adjoint_step(int model, const Grid &g, const Phys &ph, int scheme, double dt, const double *lam,
                                double *out, const double *const *Sq, const double *const *Sw, double *const *f,
                                double *const *fb, double *qbd, double *lq, double *lr2, double *lr3, double *sig,
                                cudaStream_t s) {
    if (model == 1)  // two fluids
        return adjoint_step_t<1>(g, ph, scheme, dt, lam, out, Sq, Sw, f, fb, qbd, lq, lr2, lr3, sig, s);
    return adjoint_step_t<0>(g, ph, scheme, dt, lam, out, Sq, Sw, f, fb, qbd, lq, lr2, lr3, sig, s);
}

cudaError_t launch_adjoint_prims(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                                 const double *lam, double *pbar, cudaStream_t s) {
    if (model == 1) {  // two fluids
        k_prims_adj_tf<<<blocks_for(g.ncell, 256), 256, 0, s>>>(g, ph, q, w, lam, pbar);
        return cudaGetLastError();
    }
    cudaMemsetAsync(pbar, 0, (size_t)g.plane * 11 * sizeof(double), s);
    k_prims_adj<<<blocks_for(g.ncell, 256), 256, 0, s>>>(g, ph, q, w, lam, pbar);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *x, long long n, double *out, cudaStream_t s) {
    k_sum<<<1, 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

} // namespace rmhd
