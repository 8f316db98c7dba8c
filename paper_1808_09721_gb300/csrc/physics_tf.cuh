// physics_tf.cuh -- two-fluid resistive SRMHD on the device (Sec. 2.1.2 and
// Appendix A of Wright & Hawke, arXiv:1808.09721).
//
// Conserved: D, S_i, tau (species totals), Dbar, Sbar_i, taubar (charge-to-
// mass weighted, hydrodynamic parts only), B, E, psi, phi.
// Internal primitives per species s in {e, p}: v_s (3), p_s, Z_s = rho_s h_s W_s^2.
// D_s follows from (D, Dbar) by the species split, so the flux needs no division.
//
// Implicit stage: Sbar, taubar and E (7 unknowns) have stiff sources; D, S,
// tau, Dbar, B have none; psi and phi are linear. The unknowns are scaled
// (Sbar, taubar divided by mu_ref = max |mu_s|) so that the FP32 Jacobian is
// balanced. Same precision strategy as the single fluid: FP32 Newton with
// dual-number Jacobian columns (solved by an in-place LU factorisation), then
// FP64 refinement passes with the FP32 LU factors, then consistent FP64
// primitives.
#pragma once
#include "device_math.cuh"
#include "physics_sf.cuh"
#include "rmhd_internal.h"

namespace rmhd {
namespace tf {

enum { D = 0, SX = 1, SY = 2, SZ = 3, TAU = 4, DB = 5, SBX = 6, SBY = 7, SBZ = 8, TAUB = 9,
       BX = 10, BY = 11, BZ = 12, EX = 13, EY = 14, EZ = 15, PSI = 16, PHI = 17, NC = 18 };
// per species s (offset 5 s): v (3), p, Z
enum { VX = 0, VY = 1, VZ = 2, P = 3, ZZ = 4, NW = 10 };

using sf::cross;

// Species split of Sec. 2.1.3 for a pair (total, mu-weighted):
//   X_e = (Xbar - mu_p X) / (mu_e - mu_p),  X_p = (mu_e X - Xbar) / (mu_e - mu_p).
struct Split {
    double ce_bar, ce_tot, cp_bar, cp_tot;  // X_e = ce_bar Xbar + ce_tot X ; X_p = cp_bar Xbar + cp_tot X
    __device__ __forceinline__ Split(double mu_e, double mu_p, double inv) {
        ce_bar = inv;
        ce_tot = -mu_p * inv;
        cp_bar = -inv;
        cp_tot = mu_e * inv;
    }
};

// Two-fluid flux along dir (Appendix A, Eq. twoFluid flux), T = flux arithmetic.
template <class T>
__device__ __forceinline__ void flux(const T q[NC], const T w[NW], T mu_e, T mu_p, T inv, int dir, T f[NC]) {
    const T Ds[2] = {(q[DB] - mu_p * q[D]) * inv, (mu_e * q[D] - q[DB]) * inv};
    const T mu[2] = {mu_e, mu_p};
#pragma unroll
    for (int v = 0; v < 10; ++v) f[v] = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T *ws = w + 5 * s;
        // selects (not indices computed from dir) keep the arrays in registers
        const T vd = dir == 0 ? ws[VX] : (dir == 1 ? ws[VY] : ws[VZ]);
        const T Dv = Ds[s] * vd;
        const T Zv = ws[ZZ] * vd;
        f[D] += Dv;
        f[DB] += mu[s] * Dv;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T Sij = Zv * ws[VX + i];
            if (i == dir) Sij += ws[P];
            f[SX + i] += Sij;
            f[SBX + i] += mu[s] * Sij;
        }
        f[TAUB] += mu[s] * (Zv - Dv);
    }
    const T E2B2 = q[EX] * q[EX] + q[EY] * q[EY] + q[EZ] * q[EZ] + q[BX] * q[BX] + q[BY] * q[BY] + q[BZ] * q[BZ];
    const T Ed = dir == 0 ? q[EX] : (dir == 1 ? q[EY] : q[EZ]);
    const T Bd = dir == 0 ? q[BX] : (dir == 1 ? q[BY] : q[BZ]);
    f[SX] -= q[EX] * Ed + q[BX] * Bd;
    f[SY] -= q[EY] * Ed + q[BY] * Bd;
    f[SZ] -= q[EZ] * Ed + q[BZ] * Bd;
    if (dir == 0) f[SX] += T(0.5) * E2B2; else if (dir == 1) f[SY] += T(0.5) * E2B2; else f[SZ] += T(0.5) * E2B2;
    f[TAU] = (dir == 0 ? q[SX] : (dir == 1 ? q[SY] : q[SZ])) - f[D];
    // B^i: -eps^{ijd} E_j + delta_id phi;  E^i: eps^{ijd} B_j + delta_id psi
    if (dir == 0) {
        f[BX] = q[PHI]; f[BY] = -q[EZ]; f[BZ] = q[EY];
        f[EX] = q[PSI]; f[EY] = q[BZ]; f[EZ] = -q[BY];
    } else if (dir == 1) {
        f[BX] = q[EZ]; f[BY] = q[PHI]; f[BZ] = -q[EX];
        f[EX] = -q[BZ]; f[EY] = q[PSI]; f[EZ] = q[BX];
    } else {
        f[BX] = -q[EY]; f[BY] = q[EX]; f[BZ] = q[PHI];
        f[EX] = q[BY]; f[EY] = -q[BX]; f[EZ] = q[PSI];
    }
    f[PSI] = Ed;
    f[PHI] = Bd;
}

// Source of Appendix A, written with M0 = sum mu_s^2 D_s, M1 = sum mu_s^2 D_s v_s,
// wp2 = omega_p^2 = sum mu_s^2 D_s / W_s, varrho = sum mu_s D_s, J = sum mu_s D_s v_s:
//   omega_p^2 W = M0, omega_p^2 u = M1, varrho_0 = (M0 varrho - J.M1)/wp2,
//   Sbar: M0 E + M1 x B - eta (wp2 J - varrho M1)
//   taubar: M1.E - eta (wp2 varrho - M0 varrho_0)
//   E: -J;  psi: varrho - kappa psi;  phi: -kappa phi.
template <class T, class S>
__device__ __forceinline__ void source_terms(const T Ds[2], const T v[2][3], const T sq[2], const T E[3], const S B[3],
                                             S mu_e, S mu_p, S eta, T Sb[3], T &tb, T J[3], T &varrho) {
    const S mu[2] = {mu_e, mu_p};
    T M0 = mu[0] * mu[0] * Ds[0] + mu[1] * mu[1] * Ds[1];
    T M1[3], Jv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        M1[i] = (mu[0] * mu[0]) * (Ds[0] * v[0][i]) + (mu[1] * mu[1]) * (Ds[1] * v[1][i]);
        Jv[i] = mu[0] * (Ds[0] * v[0][i]) + mu[1] * (Ds[1] * v[1][i]);
        J[i] = Jv[i];
    }
    T wp2 = (mu[0] * mu[0]) * (Ds[0] * sq[0]) + (mu[1] * mu[1]) * (Ds[1] * sq[1]);
    varrho = mu[0] * Ds[0] + mu[1] * Ds[1];
    T M1xB[3];
    cross(M1, B, M1xB);
#pragma unroll
    for (int i = 0; i < 3; ++i) Sb[i] = M0 * E[i] + M1xB[i] - eta * (wp2 * Jv[i] - varrho * M1[i]);
    T JM1 = Jv[0] * M1[0] + Jv[1] * M1[1] + Jv[2] * M1[2];
    T r0 = (M0 * varrho - JM1) * s_rcp(wp2);
    tb = (M1[0] * E[0] + M1[1] * E[1] + M1[2] * E[2]) - eta * (wp2 * varrho - M0 * r0);
}

// Recovery of the primitives of a conserved state (FP64 result).
__device__ __forceinline__ int recover(const double q[NC], const double wold[NW], const Phys &ph, double w[NW]) {
    const Split sp(ph.mu_e, ph.mu_p, ph.inv_dmu);
    const double gm1 = ph.gamma - 1.0, gam = ph.gamma;
    const double B[3] = {q[BX], q[BY], q[BZ]}, E[3] = {q[EX], q[EY], q[EZ]};
    double ExB[3];
    cross(E, B, ExB);
    double St[3] = {q[SX] - ExB[0], q[SY] - ExB[1], q[SZ] - ExB[2]};
    double taut = q[TAU] - 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    double Ds[2] = {sp.ce_bar * q[DB] + sp.ce_tot * q[D], sp.cp_bar * q[DB] + sp.cp_tot * q[D]};
    double Ss[2][3], ts[2];
    for (int i = 0; i < 3; ++i) {
        Ss[0][i] = sp.ce_bar * q[SBX + i] + sp.ce_tot * St[i];
        Ss[1][i] = sp.cp_bar * q[SBX + i] + sp.cp_tot * St[i];
    }
    ts[0] = sp.ce_bar * q[TAUB] + sp.ce_tot * taut;
    ts[1] = sp.cp_bar * q[TAUB] + sp.cp_tot * taut;
    for (int s = 0; s < 2; ++s) {
        double a = ts[s] + Ds[s];
        double S2 = Ss[s][0] * Ss[s][0] + Ss[s][1] * Ss[s][1] + Ss[s][2] * Ss[s][2];
        float p = f32_of(wold[5 * s + P]), df = -1.f;
        if (!sf::pres_solve_f32(p, f32_of(a), f32_of(S2), f32_of(Ds[s]), f32_of(gm1), f32_of(gam), df)) return sf::ST_C2P;
        double pd = f64_of(p), rdf = f64_of(1.f / df);
        pd -= sf::pres_resid(pd, a, S2, Ds[s], gm1, gam) * rdf;
        pd -= sf::pres_resid(pd, a, S2, Ds[s], gm1, gam) * rdf;
        double Z = a + pd, rZ = s_rcp(Z);
        w[5 * s + VX] = Ss[s][0] * rZ;
        w[5 * s + VY] = Ss[s][1] * rZ;
        w[5 * s + VZ] = Ss[s][2] * rZ;
        w[5 * s + P] = pd;
        w[5 * s + ZZ] = Z;
        double v2 = w[5 * s] * w[5 * s] + w[5 * s + 1] * w[5 * s + 1] + w[5 * s + 2] * w[5 * s + 2];
        if (!(pd > 0.0) || !(v2 < 1.0)) return sf::ST_C2P;
    }
    return sf::ST_OK;
}

// Source of a state with known primitives (FP64), full N_c vector.
__device__ __forceinline__ void source(const double q[NC], const double w[NW], const Phys &ph, double s[NC]) {
    const Split sp(ph.mu_e, ph.mu_p, ph.inv_dmu);
    double Ds[2] = {sp.ce_bar * q[DB] + sp.ce_tot * q[D], sp.cp_bar * q[DB] + sp.cp_tot * q[D]};
    double v[2][3], sq[2];
    for (int k = 0; k < 2; ++k) {
        for (int i = 0; i < 3; ++i) v[k][i] = w[5 * k + i];
        double om = 1.0 - (v[k][0] * v[k][0] + v[k][1] * v[k][1] + v[k][2] * v[k][2]);
        sq[k] = om * s_rsqrt(om);
    }
    const double E[3] = {q[EX], q[EY], q[EZ]}, B[3] = {q[BX], q[BY], q[BZ]};
    double Sb[3], tb, J[3], varrho;
    source_terms(Ds, v, sq, E, B, ph.mu_e, ph.mu_p, ph.eta, Sb, tb, J, varrho);
    for (int i = 0; i < NC; ++i) s[i] = 0.0;
    for (int i = 0; i < 3; ++i) {
        s[SBX + i] = Sb[i];
        s[EX + i] = -J[i];
    }
    s[TAUB] = tb;
    s[PSI] = varrho - ph.kappa * q[PSI];
    s[PHI] = -ph.kappa * q[PHI];
}

// Constant (unknown-independent) data of one stage solve, in scalar type S.
template <class S>
struct Cell {
    S D, Ds[2], Sv[3], B[3], tauB, rx[7];  // rx: scaled explicit part of the unknowns
    S mu_e, mu_p, inv, mur, imur, eta, adt, gm1, gam;
    // constants of the sources within a stage (D_s has no source): mu_s^2 D_s,
    // mu_s D_s, M0 = sum mu_s^2 D_s, varrho = sum mu_s D_s, M0 varrho
    S m2D[2], m1D[2], M0, vr, M0vr;
    // the species split of the scaled unknowns: S~_s = xs_s x_S + ct_s S~,
    // a_s = xs_s x_tau + ct_s tau~ + D_s (xs_s = +-mur / (mu_e - mu_p))
    S xs[2], ct[2];
};

// Stage residual in scaled unknowns x = (Sbar/mur, taubar/mur, E). Pressures
// p[2] must be converged for value(x) (or be one Newton step in type T).
// Outputs G (scaled), per-species S~, a, S2 are recomputed inside.
template <class T, class S>
__device__ __forceinline__ void split_x(const Cell<S> &c, const T x[7], T St2[2][3], T a[2], T S2[2]) {
    T E[3] = {x[4], x[5], x[6]};
    T ExB[3];
    cross(E, c.B, ExB);
    T St[3] = {c.Sv[0] - ExB[0], c.Sv[1] - ExB[1], c.Sv[2] - ExB[2]};
    T taut = c.tauB - S(0.5) * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int i = 0; i < 3; ++i) St2[s][i] = c.xs[s] * x[i] + c.ct[s] * St[i];
        a[s] = c.xs[s] * x[3] + (c.ct[s] * taut + c.Ds[s]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) S2[k] = St2[k][0] * St2[k][0] + St2[k][1] * St2[k][1] + St2[k][2] * St2[k][2];
}

template <class T, class S>
__device__ __forceinline__ void stage_resid(const Cell<S> &c, const T x[7], const T St2[2][3], const T a[2],
                                            const T p[2], T G[7], T v[2][3], T Z[2], T *src = nullptr,
                                            long long ps = 0) {
    T sq[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        Z[k] = a[k] + p[k];
        T rZ = s_rcp(Z[k]);
        v[k][0] = St2[k][0] * rZ;
        v[k][1] = St2[k][1] * rZ;
        v[k][2] = St2[k][2] * rZ;
        T om = S(1) - (v[k][0] * v[k][0] + v[k][1] * v[k][1] + v[k][2] * v[k][2]);
        sq[k] = om * s_rsqrt(om);
    }
    T E[3] = {x[4], x[5], x[6]};
    // the sources of Appendix A as in source_terms, with the stage's constants
    T M1[3], J[3], Sb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        M1[i] = c.m2D[0] * v[0][i] + c.m2D[1] * v[1][i];
        J[i] = c.m1D[0] * v[0][i] + c.m1D[1] * v[1][i];
    }
    const T wp2 = c.m2D[0] * sq[0] + c.m2D[1] * sq[1];
    T M1xB[3];
    cross(M1, c.B, M1xB);
#pragma unroll
    for (int i = 0; i < 3; ++i) Sb[i] = c.M0 * E[i] + M1xB[i] - c.eta * (wp2 * J[i] - c.vr * M1[i]);
    const T r0 = (c.M0vr - (J[0] * M1[0] + J[1] * M1[1] + J[2] * M1[2])) * s_rcp(wp2);
    const T tb = (M1[0] * E[0] + M1[1] * E[1] + M1[2] * E[2]) - c.eta * (wp2 * c.vr - c.M0 * r0);
    const S k1 = c.adt * c.imur;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        G[i] = (x[i] - c.rx[i]) - k1 * Sb[i];
        G[4 + i] = (x[4 + i] - c.rx[4 + i]) + c.adt * J[i];
    }
    G[3] = (x[3] - c.rx[3]) - k1 * tb;
    if (src) {  // the source entries Sbar (3), taubar, E (3) = -J at this point (7 values, ps apart)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            src[i * ps] = Sb[i];
            src[(4 + i) * ps] = -J[i];
        }
        src[3 * ps] = tb;
    }
}

// Per-thread N x N scratch matrix: a strided slice of shared memory (element
// k at p[k * stride]) or a local array (stride 1).
struct Mat {
    float *p;
    int stride;
    __device__ __forceinline__ float &operator[](int k) const { return p[k * stride]; }
};

// In-place LU factorisation with partial pivoting of an N x N FP32 matrix
// (Doolittle: L unit lower, U upper in the same storage; each pivot row swap
// is applied to the stored rows and its row index kept in 3 bits of piv; the
// diagonal holds the reciprocals of U's pivots).
template <int N>
__device__ __forceinline__ bool lu_factor(Mat m, unsigned &piv) {
    static_assert(N <= 8, "3 bits per pivot");
    piv = 0u;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        int pr = c;
        float best = fabsf(m[c * N + c]);
#pragma unroll
        for (int r = c + 1; r < N; ++r)
            if (fabsf(m[r * N + c]) > best) { best = fabsf(m[r * N + c]); pr = r; }
        if (!(best > 0.f) || !isfinite(best)) return false;
        piv |= (unsigned)pr << (3 * c);
        if (pr != c)
            for (int k = 0; k < N; ++k) { const float t = m[c * N + k]; m[c * N + k] = m[pr * N + k]; m[pr * N + k] = t; }
        const float id = 1.f / m[c * N + c];
        m[c * N + c] = id;
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            const float f = m[r * N + c] * id;
            m[r * N + c] = f;
#pragma unroll
            for (int k = c + 1; k < N; ++k) m[r * N + k] -= f * m[c * N + k];
        }
    }
    return true;
}

// b <- A^{-1} b from lu_factor's storage.
template <int N>
__device__ __forceinline__ void lu_solve(Mat m, unsigned piv, float b[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const int pr = (piv >> (3 * c)) & 7;
#pragma unroll
        for (int r = c + 1; r < N; ++r)
            if (r == pr) { const float t = b[c]; b[c] = b[r]; b[r] = t; }
    }
#pragma unroll
    for (int i = 1; i < N; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) b[i] -= m[i * N + j] * b[j];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
#pragma unroll
        for (int j = i + 1; j < N; ++j) b[i] -= m[i * N + j] * b[j];
        b[i] *= m[i * N + i];
    }
}

// Magnitude of the terms of the stage residual G at (x, v) in FP32: the
// round-off scale of G (norms bound the products inside the sources).
__device__ __forceinline__ float resid_scale(const Cell<float> &cf, const float x[7], const float v[2][3]) {
    const float mu[2] = {cf.mu_e, cf.mu_p};
    float M0 = 0.f, M1n = 0.f, Jn = 0.f, vr = 0.f;
    for (int sp = 0; sp < 2; ++sp) {
        float vn = fabsf(v[sp][0]) + fabsf(v[sp][1]) + fabsf(v[sp][2]);
        M0 += mu[sp] * mu[sp] * cf.Ds[sp];
        M1n += mu[sp] * mu[sp] * cf.Ds[sp] * vn;
        Jn += fabsf(mu[sp]) * cf.Ds[sp] * vn;
        vr += fabsf(mu[sp]) * cf.Ds[sp];
    }
    const float En = fabsf(x[4]) + fabsf(x[5]) + fabsf(x[6]);
    const float Bn = fabsf(cf.B[0]) + fabsf(cf.B[1]) + fabsf(cf.B[2]);
    const float src = M0 * En + M1n * Bn + cf.eta * (M0 * Jn + vr * M1n);
    float gs = 1e-30f;
    for (int i = 0; i < 7; ++i) gs = fmaxf(gs, fabsf(x[i]) + fabsf(cf.rx[i]));
    gs = fmaxf(gs, cf.adt * cf.imur * src);
    gs = fmaxf(gs, cf.adt * Jn);
    return gs;
}

struct StageConst {
    double adt, cpsi;
    int maxpass;               // FP64 refinement passes at most (1..8)
    unsigned long long *hist;  // if not null: histograms of FP32 iterations [32] and FP64 passes [8]
};

// The FP64 data of a cell's stage solve from its explicit part r (variables
// ps apart).
__device__ __forceinline__ void load_cell(Cell<double> &c, const double *rp, long long ps, const Split &sp,
                                          const StageConst &k, const Phys &ph) {
    c.D = rp[D * ps];
    const double Db = rp[DB * ps];
    c.Ds[0] = sp.ce_bar * Db + sp.ce_tot * c.D;
    c.Ds[1] = sp.cp_bar * Db + sp.cp_tot * c.D;
    for (int i = 0; i < 3; ++i) { c.Sv[i] = rp[(SX + i) * ps]; c.B[i] = rp[(BX + i) * ps]; }
    c.tauB = rp[TAU * ps] - 0.5 * (c.B[0] * c.B[0] + c.B[1] * c.B[1] + c.B[2] * c.B[2]);
    c.mu_e = ph.mu_e; c.mu_p = ph.mu_p; c.inv = ph.inv_dmu;
    c.mur = ph.mur;
    c.imur = ph.imur;
    c.eta = ph.eta;
    c.adt = k.adt; c.gm1 = ph.gamma - 1.0; c.gam = ph.gamma;
    for (int i = 0; i < 3; ++i) { c.rx[i] = rp[(SBX + i) * ps] * c.imur; c.rx[4 + i] = rp[(EX + i) * ps]; }
    c.rx[3] = rp[TAUB * ps] * c.imur;
    for (int s = 0; s < 2; ++s) {
        const double mu = s == 0 ? ph.mu_e : ph.mu_p;
        c.m1D[s] = mu * c.Ds[s];
        c.m2D[s] = mu * c.m1D[s];
    }
    c.M0 = c.m2D[0] + c.m2D[1];
    c.vr = c.m1D[0] + c.m1D[1];
    c.M0vr = c.M0 * c.vr;
    c.xs[0] = c.mur * c.inv;
    c.xs[1] = -c.xs[0];
    c.ct[0] = -c.mu_p * c.inv;
    c.ct[1] = c.mu_e * c.inv;
}

// Solve one implicit stage for one cell (two fluids). rp: the cell's explicit
// part (18 FP64 variables, ps apart); wwarm: its warm-start primitives (10,
// ps apart). Writes q (18, through qp) and w (10, through wp), and, if srcp
// is not null, the source entries Sbar (3), taubar, E (3) at the result (7,
// ps apart; Appendix A). Jm is the caller's 7 x 7 FP32 scratch for the
// Jacobian and its LU factors. The
// FP64 cell data are built again after the FP32 Newton phase rather than held
// in registers through it.
template <int NREF, bool STATS = false>
__device__ int stage_solve(const double *rp, long long ps, const double *wwarm, const StageConst &k,
                           const Phys &ph, double *qp, double *wp, Mat Jm, double *srcp = nullptr) {
    const Split sp(ph.mu_e, ph.mu_p, ph.inv_dmu);
    const double gm1 = ph.gamma - 1.0, gam = ph.gamma;

    Cell<float> cf;
    {
        Cell<double> c;
        load_cell(c, rp, ps, sp, k, ph);
        cf.D = f32_of(c.D); cf.Ds[0] = f32_of(c.Ds[0]); cf.Ds[1] = f32_of(c.Ds[1]);
        for (int i = 0; i < 3; ++i) { cf.Sv[i] = f32_of(c.Sv[i]); cf.B[i] = f32_of(c.B[i]); }
        cf.tauB = f32_of(c.tauB);
        for (int i = 0; i < 7; ++i) cf.rx[i] = f32_of(c.rx[i]);
        cf.mu_e = f32_of(c.mu_e); cf.mu_p = f32_of(c.mu_p); cf.inv = f32_of(c.inv); cf.mur = f32_of(c.mur);
        cf.imur = f32_of(c.imur); cf.eta = f32_of(c.eta); cf.adt = f32_of(c.adt); cf.gm1 = f32_of(gm1);
        cf.gam = f32_of(gam);
        for (int s = 0; s < 2; ++s) { cf.m2D[s] = f32_of(c.m2D[s]); cf.m1D[s] = f32_of(c.m1D[s]); }
        cf.M0 = f32_of(c.M0); cf.vr = f32_of(c.vr); cf.M0vr = f32_of(c.M0vr);
        for (int s = 0; s < 2; ++s) { cf.xs[s] = f32_of(c.xs[s]); cf.ct[s] = f32_of(c.ct[s]); }
        // source-free components equal r; psi and phi in closed form (varrho = Dbar has no source)
        for (int v : {D, SX, SY, SZ, TAU, DB, BX, BY, BZ}) qp[v * ps] = rp[v * ps];
        for (int i = 0; i < 3; ++i) qp[(EX + i) * ps] = rp[(EX + i) * ps];  // replaced by the root
        for (int i = 0; i < 4; ++i) qp[(SBX + i) * ps] = rp[(SBX + i) * ps];  // replaced by the root
        qp[PSI * ps] = (rp[PSI * ps] + k.adt * rp[DB * ps]) * k.cpsi;
        qp[PHI * ps] = rp[PHI * ps] * k.cpsi;
    }

    float scale = 1e-30f;
    for (int i = 0; i < 7; ++i) scale = fmaxf(scale, fabsf(cf.rx[i]));

    // ---- FP32 Newton
    float x[7], p[2] = {f32_of(wwarm[P * ps]), f32_of(wwarm[(5 + P) * ps])}, dfdp[2] = {-1.f, -1.f};
    for (int i = 0; i < 7; ++i) x[i] = cf.rx[i];
    float St2[2][3], a[2], S2[2], G[7], v[2][3], Z[2];
    split_x(cf, x, St2, a, S2);
    for (int s = 0; s < 2; ++s)
        if (!sf::pres_solve_f32(p[s], a[s], S2[s], cf.Ds[s], cf.gm1, cf.gam, dfdp[s])) return sf::ST_C2P;
    stage_resid(cf, x, St2, a, p, G, v, Z);
    float gn = 0.f;
    for (int i = 0; i < 7; ++i) gn = fmaxf(gn, fabsf(G[i]));

    float dpdx[2][7];
    bool have_jac = false;
    unsigned piv = 0u;
    int nit = 0;
    for (int it = 0; it < 30; ++it) {
        nit = it + 1;
        for (int kc = 0; kc < 7; ++kc) {
            Dual<float> xd[7];
            for (int i = 0; i < 7; ++i) xd[i] = Dual<float>(x[i], i == kc ? 1.f : 0.f);
            Dual<float> Std[2][3], ad[2], S2d[2], pd[2], Gd[7], vd[2][3], Zd[2];
            split_x(cf, xd, Std, ad, S2d);
            for (int s = 0; s < 2; ++s) {
                Dual<float> ps(p[s]);
                Dual<float> fs = sf::pres_resid(ps, ad[s], S2d[s], cf.Ds[s], cf.gm1, cf.gam);
                pd[s] = Dual<float>(p[s], -fs.d / dfdp[s]);
                dpdx[s][kc] = pd[s].d;
            }
            stage_resid(cf, xd, Std, ad, pd, Gd, vd, Zd);
            for (int i = 0; i < 7; ++i) Jm[i * 7 + kc] = Gd[i].d;
        }
        if (!lu_factor<7>(Jm, piv)) return sf::ST_NEWTON;
        have_jac = true;
        float dx[7], dn = 0.f, xn = scale;
        for (int i = 0; i < 7; ++i) dx[i] = G[i];
        lu_solve<7>(Jm, piv, dx);
        for (int i = 0; i < 7; ++i) {
            dn = fmaxf(dn, fabsf(dx[i]));
            xn = fmaxf(xn, fabsf(x[i]));
        }
        if (dn <= 2e-7f * xn) break;
        // |G| at the FP32 noise floor: the FP64 passes take over
        if (gn <= 1e-6f * resid_scale(cf, x, v)) break;
        float t = 1.f;
        bool accepted = false;
        for (int ls = 0; ls < 8; ++ls) {
            float xt[7], pt[2] = {p[0], p[1]}, dft[2] = {dfdp[0], dfdp[1]}, Gt[7], vt[2][3], Zt[2];
            float St2t[2][3], at[2], S2t[2];
            for (int i = 0; i < 7; ++i) xt[i] = x[i] - t * dx[i];
            split_x(cf, xt, St2t, at, S2t);
            bool ok = sf::pres_solve_f32(pt[0], at[0], S2t[0], cf.Ds[0], cf.gm1, cf.gam, dft[0]) &&
                      sf::pres_solve_f32(pt[1], at[1], S2t[1], cf.Ds[1], cf.gm1, cf.gam, dft[1]);
            if (ok) {
                stage_resid(cf, xt, St2t, at, pt, Gt, vt, Zt);
                float gt = 0.f;
                for (int i = 0; i < 7; ++i) gt = fmaxf(gt, fabsf(Gt[i]));
                if (gt < gn || t < 0.02f) {
                    for (int i = 0; i < 7; ++i) { x[i] = xt[i]; G[i] = Gt[i]; }
                    for (int i = 0; i < 3; ++i) { v[0][i] = vt[0][i]; v[1][i] = vt[1][i]; }
                    p[0] = pt[0]; p[1] = pt[1]; dfdp[0] = dft[0]; dfdp[1] = dft[1];
                    gn = gt;
                    accepted = true;
                    break;
                }
            }
            t *= 0.5f;
        }
        if (!accepted) break;
    }
    if (!have_jac) return sf::ST_NEWTON;

    // ---- FP64 refinement passes (as for one fluid: the evaluation point where
    // |G| reaches round-off of the magnitude of G's terms is the result, with
    // its own primitives; extra passes, up to 8, only where needed)
    const float gs = resid_scale(cf, x, v);  // round-off scale of G
    Cell<double> c;  // read again (the stores above keep the first loads from being reused)
    load_cell(c, rp, ps, sp, k, ph);
    double xd[7], pdd[2] = {f64_of(p[0]), f64_of(p[1])};
    const double rdf[2] = {f64_of(1.f / dfdp[0]), f64_of(1.f / dfdp[1])};
    for (int i = 0; i < 7; ++i) xd[i] = f64_of(x[i]);
    double St64[2][3], a64[2], S264[2], G64[7], v64[2][3], Z64[2];
    float gres = 0.f;  // |G| in FP32 (f32_of maps a NaN to an infinity)
    int pass = 0;
#pragma unroll 1
    for (; pass < 8; ++pass) {  // constant trip count; the cap k.maxpass breaks below
        split_x(c, xd, St64, a64, S264);
        for (int s = 0; s < 2; ++s) pdd[s] -= sf::pres_resid(pdd[s], a64[s], S264[s], c.Ds[s], gm1, gam) * rdf[s];
        // every pass writes the sources at its point: the last pass's stay
        stage_resid(c, xd, St64, a64, pdd, G64, v64, Z64, srcp, ps);
        float dx[7];
        gres = 0.f;
        for (int i = 0; i < 7; ++i) {
            dx[i] = f32_of(G64[i]);
            gres = fmaxf(gres, fabsf(dx[i]));
        }
        if (pass >= NREF - 1 && gres * 1e12f <= gs) break;
        if (pass == 7 || pass == k.maxpass - 1) break;
        lu_solve<7>(Jm, piv, dx);
        for (int s = 0; s < 2; ++s) {
            float dp = 0.f;
            for (int i = 0; i < 7; ++i) dp += dpdx[s][i] * dx[i];
            pdd[s] -= f64_of(dp);
        }
        for (int i = 0; i < 7; ++i) xd[i] -= f64_of(dx[i]);
    }
    bool ok = true;
    for (int s = 0; s < 2; ++s) {
        wp[(5 * s + VX) * ps] = v64[s][0];
        wp[(5 * s + VY) * ps] = v64[s][1];
        wp[(5 * s + VZ) * ps] = v64[s][2];
        wp[(5 * s + P) * ps] = pdd[s];
        wp[(5 * s + ZZ) * ps] = Z64[s];
        ok = ok && pdd[s] > 0.0 && isfinite(Z64[s]);
    }
    for (int i = 0; i < 3; ++i) {
        qp[(SBX + i) * ps] = xd[i] * c.mur;
        qp[(EX + i) * ps] = xd[4 + i];
    }
    qp[TAUB * ps] = xd[3] * c.mur;
    ok = ok && gres * 1e9f <= gs;
    if constexpr (STATS) sf::count_solve(k.hist, nit, pass + 1, ok ? 0 : 3);
    if (!ok) return sf::ST_NEWTON;
    return sf::ST_OK;
}

} // namespace tf
} // namespace rmhd
