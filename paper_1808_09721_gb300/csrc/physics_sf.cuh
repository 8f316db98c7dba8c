// physics_sf.cuh -- single-fluid resistive SRMHD on the device (Sec. 2.1.1 of
// Wright & Hawke, arXiv:1808.09721): primitive recovery (Sec. 2.1.3), Ohm's-law
// current, flux along x or y, and the per-cell implicit stage of the IMEX
// scheme (Eq. implicit stage).
//
// Implicit stage q = r + a dt Psi(q): D, S, tau, B and varrho have no source
// and equal r; psi and phi are linear in themselves and solved in closed form;
// E (3 unknowns) solves G(E) = E - r_E + a dt J(E) = 0, where J needs the
// primitives of q(E) and hence a pressure root per evaluation.
//
// Precision strategy (GB300: FP64 is ~1/67 of FP32 throughput):
//   1. Newton on G in FP32 until the FP32 residual stalls (~1e-7 relative).
//      Jacobian columns come from forward-mode duals through the same code,
//      the pressure root's derivative by the implicit-function theorem.
//   2. FP64 refinement passes (two for almost every cell): evaluate G in FP64
//      (one FP64 Newton step of the pressure root per pass, started from a
//      first-order prediction) and correct E with the FP32 inverse Jacobian.
//      Each pass gains ~6-7 digits. The first evaluation point (from the
//      second on) where |G| is at round-off of the magnitude of G's terms
//      (relative 1e-12, tighter in stiff cells) is returned with its own
//      primitives, so E and v are consistent.
#pragma once
#include "device_math.cuh"

namespace rmhd {
namespace sf {

enum { D = 0, SX = 1, SY = 2, SZ = 3, TAU = 4, BX = 5, BY = 6, BZ = 7, EX = 8, EY = 9, EZ = 10, RHOE = 11, PSI = 12, PHI = 13, NC = 14 };
// internal primitives kept per cell: velocity, pressure and Lorentz factor
enum { VX = 0, VY = 1, VZ = 2, P = 3, LOR = 4, NW = 5 };

template <class A, class B, class C>
__device__ __forceinline__ void cross(const A a[3], const B b[3], C c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Pressure-root residual for one species with hydrodynamic data:
// a = tau~ + D, S2 = |S~|^2. With Z = a + p = rho h W^2 and v^2 = S2/Z^2,
//   f(p) = (Gamma-1) [Z - S2/Z - D sqrt(1 - v^2)] - Gamma p,
// which vanishes exactly when p = (Gamma-1) rho eps (Sec. 2.1 EOS).
template <class T, class S>
__device__ __forceinline__ T pres_resid(T p, T a, T S2, S Dd, S gm1, S gam) {
    T Z = a + p;
    T rZ = s_rcp(Z);
    T v2 = S2 * rZ * rZ;
    T om = S(1) - v2;
    T sq = om * s_rsqrt(om);
    return gm1 * (Z - S2 * rZ - Dd * sq) - gam * p;
}

// FP32 Newton-bisection solve of the pressure root from the guess p.
// Returns false if the data admit no root (|S~| >= tau~ + D or D <= 0).
// On return p is converged (to ~1e-6 relative) and dfdp the slope there.
__device__ __forceinline__ bool pres_solve_f32(float &p, float a, float S2, float Dd, float gm1, float gam, float &dfdp) {
    if (!(Dd > 0.f) || !(a * a > S2) || !(a > 0.f)) return false;
    float lo = 0.f, hi = gm1 * a;
    if (!(p > lo && p < hi)) p = 0.5f * hi;
    for (int it = 0; it < 60; ++it) {
        float Z = a + p;
        float rZ = s_rcp(Z);
        float v2 = S2 * rZ * rZ;
        float om = 1.f - v2;
        float W = s_rsqrt(om);
        float sq = om * W;
        float f = gm1 * (Z - S2 * rZ - Dd * sq) - gam * p;
        float df = gm1 * (1.f + v2 - Dd * v2 * rZ * W) - gam;
        dfdp = df;
        if (f > 0.f) lo = p; else hi = p;
        float pn = p - f / df;
        if (!(pn > lo && pn < hi)) pn = 0.5f * (lo + hi);
        float dp = fabsf(pn - p);
        p = pn;
        if (dp <= 2e-7f * p || hi - lo <= 2e-7f * hi) return true;
    }
    return true;
}

// EM split of Sec. 2.1.3: S~ = S - E x B, tau~ = tau - (E^2 + B^2)/2.
// tauB = tau - B^2/2 is precomputed; a = tau~ + D; S2 = |S~|^2.
template <class T, class S>
__device__ __forceinline__ void em_split(const T E[3], const S Sv[3], const S B[3], S tauB, S Dd, T St[3], T &a, T &S2) {
    T ExB[3];
    cross(E, B, ExB);
    St[0] = Sv[0] - ExB[0];
    St[1] = Sv[1] - ExB[1];
    St[2] = Sv[2] - ExB[2];
    T E2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
    a = (tauB + Dd) - S(0.5) * E2;
    S2 = St[0] * St[0] + St[1] * St[1] + St[2] * St[2];
}

// Stage residual at E given a converged pressure p:
//   v = S~/(a + p), W = (1 - v^2)^(-1/2),
//   J = varrho v + W sigma [E + v x B - (v.E) v]   (Ohm's law, Sec. 2.1.1),
//   G = E - r_E + a dt J.
template <class T, class S>
__device__ __forceinline__ void stage_resid(const T E[3], T p, const T St[3], T a, const S B[3], const S rE[3], S rhoe,
                                            S adt, S sig, T G[3], T v[3], T &W) {
    T rZ = s_rcp(a + p);
    v[0] = St[0] * rZ;
    v[1] = St[1] * rZ;
    v[2] = St[2] * rZ;
    T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    W = s_rsqrt(S(1) - v2);
    T vxB[3];
    cross(v, B, vxB);
    T vE = v[0] * E[0] + v[1] * E[1] + v[2] * E[2];
    T Ws = W * sig;
    for (int i = 0; i < 3; ++i) {
        T u = E[i] + vxB[i] - vE * v[i];
        T J = rhoe * v[i] + Ws * u;
        G[i] = (E[i] - rE[i]) + adt * J;
    }
}

// The EM split and the stage residual of the FP64 passes, with the per-cell
// constants folded: tD = tau - B^2/2 + D (a = tD - E^2/2), arho = a dt varrho,
// asig = a dt sigma,
//   G = E - r_E + arho v + asig W u,  u = E + v x B - (v.E) v
// (u is returned: the current at the result is varrho v + sigma W u).
__device__ __forceinline__ void em_split_folded(const double E[3], const double Sv[3], const double B[3], double tD,
                                                double St[3], double &a, double &S2) {
    double ExB[3];
    cross(E, B, ExB);
    St[0] = Sv[0] - ExB[0];
    St[1] = Sv[1] - ExB[1];
    St[2] = Sv[2] - ExB[2];
    a = tD - 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
    S2 = St[0] * St[0] + St[1] * St[1] + St[2] * St[2];
}
__device__ __forceinline__ void stage_resid_folded(const double E[3], double p, const double St[3], double a,
                                                   const double B[3], const double rE[3], double arho, double asig,
                                                   double G[3], double v[3], double &W, double u[3]) {
    const double rZ = s_rcp(a + p);
    v[0] = St[0] * rZ;
    v[1] = St[1] * rZ;
    v[2] = St[2] * rZ;
    const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    W = s_rsqrt(1.0 - v2);
    double vxB[3];
    cross(v, B, vxB);
    const double vE = v[0] * E[0] + v[1] * E[1] + v[2] * E[2];
    const double aW = asig * W;
    for (int i = 0; i < 3; ++i) {
        u[i] = E[i] + vxB[i] - vE * v[i];
        G[i] = fma(aW, u[i], fma(arho, v[i], E[i] - rE[i]));
    }
}

// 3x3 inverse by cofactors (FP32). Returns false if singular.
__device__ __forceinline__ bool inv3(const float m[9], float inv[9]) {
    float c0 = m[4] * m[8] - m[5] * m[7];
    float c1 = m[5] * m[6] - m[3] * m[8];
    float c2 = m[3] * m[7] - m[4] * m[6];
    float det = m[0] * c0 + m[1] * c1 + m[2] * c2;
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    float id = 1.f / det;
    inv[0] = c0 * id;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    inv[3] = c1 * id;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    inv[6] = c2 * id;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) * id;
    return true;
}

// Magnitude of the terms of the stage residual G at (E, v, W) in FP32: the
// round-off scale of G. The products inside v x B and v.E are bounded one by
// one, because in a near-static cell the two products of a cross-product
// component can cancel to ~1e-9 of their size.
__device__ __forceinline__ float resid_scale(const float E[3], const float rE[3], const float v[3], const float B[3],
                                             float W, float rhoe, float adt, float sig) {
    const float av[3] = {fabsf(v[0]), fabsf(v[1]), fabsf(v[2])};
    const float aB[3] = {fabsf(B[0]), fabsf(B[1]), fabsf(B[2])};
    const float vEn = av[0] * fabsf(E[0]) + av[1] * fabsf(E[1]) + av[2] * fabsf(E[2]);
    float gs = 1e-30f;
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, l = (i + 2) % 3;
        const float cr = av[j] * aB[l] + av[l] * aB[j];
        gs = fmaxf(gs, fabsf(E[i]) + fabsf(rE[i]) + adt * (fabsf(rhoe) * av[i] + sig * W * (fabsf(E[i]) + cr + vEn * av[i])));
    }
    return gs;
}

// Status codes recorded per cell (match the library's error codes).
enum { ST_OK = 0, ST_NEWTON = -3, ST_C2P = -4 };

struct StageConst {
    double adt;   // a_ii dt
    double cpsi;  // 1 / (1 + adt kappa)
    double sigma, gamma;
    int maxpass;                // FP64 refinement passes at most (1..8)
    unsigned long long *hist;   // if not null: histograms of FP32 iterations [32] and FP64 passes [8]
};

// Adds one solve to the histograms: by FP32 Newton iterations, by FP64
// passes, and by the start that converged (start 0, 1, 2; 3: none did).
__device__ __forceinline__ void count_solve(unsigned long long *hist, int nit, int npass, int start) {
    if (!hist) return;
    atomicAdd(&hist[nit < 31 ? nit : 31], 1ULL);
    atomicAdd(&hist[32 + npass - 1], 1ULL);
    atomicAdd(&hist[40 + start], 1ULL);
}

// Solve one implicit stage for one cell. rp: the cell's explicit part (14
// FP64 variables, ps apart); p_warm: pressure guess. Writes the cell's q (14,
// through qp) and w = (v, p, W) (through wp), ps apart. NREF FP64 passes.
// The FP64 inputs of the refinement passes are read again after the FP32
// Newton phase instead of being held in registers through it (they are in
// L1), which keeps the kernel at a higher occupancy. STATS adds the solve to
// the iteration histogram k.hist; it is a template switch rather than a null
// test because the live counters lengthen the latency-bound code even when
// nothing is counted.
//
// Starts (the root is the same whichever converges; only the path differs):
//   0. E = r_E;
//   1. the ideal-MHD limit E = -v x B with v recovered at E = r_E (the
//      sigma -> infinity root, Sec. 2.1.1), if start 0 fails;
//   2. continuation in a dt: the stage solved for a dt / 64, a dt / 32, ...,
//      a dt in FP32, each from the previous root, if start 1 fails too.
// A start fails on a singular FP32 Jacobian, an FP32 pressure root that does
// not exist, or FP64 passes that do not reach the acceptance test.
// stage_solve runs start 0 and returns ST_NEWTON when it fails; the kernels
// then hand the cell to stage_restarts (starts 1 and 2) in a separate launch,
// which keeps the register allocation of the common path unchanged.
template <int NREF, bool STATS = false>
__device__ __forceinline__ int stage_solve(const double *rp, long long ps, double p_warm, const StageConst &k,
                                           double *qp, double *wp, double *jp = nullptr) {
    const double gm1 = k.gamma - 1.0, gam = k.gamma;
    double tauB;
    float Bf[3], Sf[3], rEf[3], tauBf, Df, rhoef;
    {
        const double B[3] = {rp[BX * ps], rp[BY * ps], rp[BZ * ps]};
        const double Sv[3] = {rp[SX * ps], rp[SY * ps], rp[SZ * ps]};
        const double tau = rp[TAU * ps], Dd = rp[D * ps], rhoe = rp[RHOE * ps];
        tauB = tau - 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        for (int i = 0; i < 3; ++i) {
            const double rEi = rp[(EX + i) * ps];
            Bf[i] = f32_of(B[i]);
            Sf[i] = f32_of(Sv[i]);
            rEf[i] = f32_of(rEi);
            qp[(EX + i) * ps] = rEi;  // replaced by the root; left as r_E if the solve fails
        }
        tauBf = f32_of(tauB);
        Df = f32_of(Dd);
        rhoef = f32_of(rhoe);
        // source-free components equal r; psi and phi in closed form
        qp[D * ps] = Dd;
        qp[TAU * ps] = tau;
        qp[RHOE * ps] = rhoe;
        for (int i = 0; i < 3; ++i) {
            qp[(SX + i) * ps] = Sv[i];
            qp[(BX + i) * ps] = B[i];
        }
        qp[PSI * ps] = (rp[PSI * ps] + k.adt * rhoe) * k.cpsi;
        qp[PHI * ps] = rp[PHI * ps] * k.cpsi;
    }

    // ---- FP32 Newton
    const float adtf = f32_of(k.adt), sigf = f32_of(k.sigma), gm1f = f32_of(gm1), gamf = f32_of(gam);
    const float scale = fmaxf(fmaxf(fabsf(rEf[0]), fabsf(rEf[1])), fmaxf(fabsf(rEf[2]), 1e-30f));

    float E[3] = {rEf[0], rEf[1], rEf[2]};
    float p = f32_of(p_warm), dfdp = -1.f;
    float G[3], v[3], W, St[3], a, S2;
    em_split(E, Sf, Bf, tauBf, Df, St, a, S2);
    if (!pres_solve_f32(p, a, S2, Df, gm1f, gamf, dfdp)) return ST_C2P;
    stage_resid(E, p, St, a, Bf, rEf, rhoef, adtf, sigf, G, v, W);
    float gn = fmaxf(fmaxf(fabsf(G[0]), fabsf(G[1])), fabsf(G[2]));

    float Minv[9], dpdE[3];
    bool have_jac = false;
    int nit = 0;
    for (int it = 0; it < 24; ++it) {
        nit = it + 1;
        // Jacobian columns dG/dE_k with duals; dp/dE_k by the implicit-function theorem
        float Jm[9];
        for (int kc = 0; kc < 3; ++kc) {
            Dual<float> Ed[3] = {Dual<float>(E[0], kc == 0), Dual<float>(E[1], kc == 1), Dual<float>(E[2], kc == 2)};
            Dual<float> Std[3], ad, S2d;
            em_split(Ed, Sf, Bf, tauBf, Df, Std, ad, S2d);
            Dual<float> pd(p);
            Dual<float> fd = pres_resid(pd, ad, S2d, Df, gm1f, gamf);
            pd = Dual<float>(p, -fd.d / dfdp);
            dpdE[kc] = pd.d;
            Dual<float> Gd[3], vd[3], Wd;
            stage_resid(Ed, pd, Std, ad, Bf, rEf, rhoef, adtf, sigf, Gd, vd, Wd);
            Jm[0 + kc] = Gd[0].d;
            Jm[3 + kc] = Gd[1].d;
            Jm[6 + kc] = Gd[2].d;
        }
        if (!inv3(Jm, Minv)) return ST_NEWTON;
        have_jac = true;
        float dE[3];
        for (int i = 0; i < 3; ++i) dE[i] = Minv[3 * i] * G[0] + Minv[3 * i + 1] * G[1] + Minv[3 * i + 2] * G[2];
        float dn = fmaxf(fmaxf(fabsf(dE[0]), fabsf(dE[1])), fabsf(dE[2]));
        if (dn <= 2e-7f * fmaxf(scale, fmaxf(fmaxf(fabsf(E[0]), fabsf(E[1])), fabsf(E[2])))) break;
        // |G| at the FP32 noise floor (p and v carry ~2e-7 relative error):
        // further FP32 steps cannot improve E; the FP64 passes take over
        if (gn <= 1e-6f * resid_scale(E, rEf, v, Bf, W, rhoef, adtf, sigf)) break;
        // backtracking on |G|_inf
        float t = 1.f;
        bool accepted = false;
        for (int ls = 0; ls < 8; ++ls) {
            float Et[3] = {E[0] - t * dE[0], E[1] - t * dE[1], E[2] - t * dE[2]};
            float pt = p, dft = dfdp, Gt[3], vt[3], Wt, Stt[3], at, S2t;
            em_split(Et, Sf, Bf, tauBf, Df, Stt, at, S2t);
            if (pres_solve_f32(pt, at, S2t, Df, gm1f, gamf, dft)) {
                stage_resid(Et, pt, Stt, at, Bf, rEf, rhoef, adtf, sigf, Gt, vt, Wt);
                float gt = fmaxf(fmaxf(fabsf(Gt[0]), fabsf(Gt[1])), fabsf(Gt[2]));
                if (gt < gn || (t < 0.02f && gt <= 1.5f * gn)) {
                    E[0] = Et[0]; E[1] = Et[1]; E[2] = Et[2];
                    p = pt; dfdp = dft; G[0] = Gt[0]; G[1] = Gt[1]; G[2] = Gt[2];
                    v[0] = vt[0]; v[1] = vt[1]; v[2] = vt[2]; W = Wt;
                    gn = gt;
                    accepted = true;
                    break;
                }
            }
            t *= 0.5f;
        }
        if (!accepted) break;  // FP32 noise floor: hand over to the FP64 passes
    }
    if (!have_jac) return ST_NEWTON;

    // ---- FP64 refinement passes. Pass k evaluates G in FP64 at E_k (one FP64
    // pressure step, started from a first-order prediction) and forms the
    // correction dE_k with the FP32 inverse Jacobian. The evaluation point at
    // which |G| reaches round-off of the magnitude of G's terms (at least the
    // NREF-th) is the result, with its own primitives (J amplifies any E/v
    // mismatch by sigma). Cells that need it take extra passes (up to 8).
    const float gs = resid_scale(E, rEf, v, Bf, W, rhoef, adtf, sigf);  // round-off scale of G
    // Acceptance |G| <= tol gs. The explicit stages evaluate J = sigma W (E + v x B
    // - (v.E) v) at the accepted E, which multiplies an E error by ~sigma dt W,
    // while G's own terms carry a dt sigma W: for stiff cells (a dt sigma W >> 1)
    // the tolerance shrinks by that factor, down to a few units of FP64
    // round-off of G's terms. Non-stiff cells keep 1e-12.
    const float itol = 1.f / fmaxf(1e-12f * s_rcp(1.f + adtf * sigf * W), 1e-15f);
    // FP64 inputs, read again (the stores above keep the compiler from reusing
    // the first loads' registers)
    const double B[3] = {rp[BX * ps], rp[BY * ps], rp[BZ * ps]};
    const double Sv[3] = {rp[SX * ps], rp[SY * ps], rp[SZ * ps]};
    const double rE[3] = {rp[EX * ps], rp[EY * ps], rp[EZ * ps]};
    const double Dd = rp[D * ps], rhoe = rp[RHOE * ps];
    const double tD = tauB + Dd, arho = k.adt * rhoe, asig = k.adt * k.sigma;
    double Ed[3] = {f64_of(E[0]), f64_of(E[1]), f64_of(E[2])};
    double pdd = f64_of(p);
    const double rdf = f64_of(1.f / dfdp);
    double St64[3], a64, S264, G64[3], v64[3], W64, u64[3];
    float gres = 0.f;
    bool pconv = false;
    int pass = 0;
    for (; pass < 8; ++pass) {  // constant trip count; the cap k.maxpass breaks below
        em_split_folded(Ed, Sv, B, tD, St64, a64, S264);
        const double dp = pres_resid(pdd, a64, S264, Dd, gm1, gam) * rdf;
        pdd -= dp;
        pconv = f32_of(fabs(dp)) <= 1e-6f * f32_of(pdd);
        stage_resid_folded(Ed, pdd, St64, a64, B, rE, arho, asig, G64, v64, W64, u64);
        float Gf[3] = {f32_of(G64[0]), f32_of(G64[1]), f32_of(G64[2])};
        // |G| in FP32 from the copy the correction uses (f32_of maps a NaN to an
        // infinity, so a non-finite G fails the tests)
        gres = fmaxf(fmaxf(fabsf(Gf[0]), fabsf(Gf[1])), fabsf(Gf[2]));
        if (pass >= NREF - 1 && gres * itol <= gs && pconv) break;
        float dE[3];
        for (int i = 0; i < 3; ++i) dE[i] = Minv[3 * i] * Gf[0] + Minv[3 * i + 1] * Gf[1] + Minv[3 * i + 2] * Gf[2];
        if (pass == 7 || pass == k.maxpass - 1) break;
        // first-order prediction of the pressure at the corrected E
        pdd -= f64_of(dpdE[0] * dE[0] + dpdE[1] * dE[1] + dpdE[2] * dE[2]);
        Ed[0] -= f64_of(dE[0]);
        Ed[1] -= f64_of(dE[1]);
        Ed[2] -= f64_of(dE[2]);
    }
    wp[VX * ps] = v64[0];
    wp[VY * ps] = v64[1];
    wp[VZ * ps] = v64[2];
    wp[P * ps] = pdd;
    wp[LOR * ps] = W64;
    qp[EX * ps] = Ed[0];
    qp[EY * ps] = Ed[1];
    qp[EZ * ps] = Ed[2];
    if (jp) {  // for the flux pass: Ohm's-law current (as current() forms it), Z, p + (E^2 + B^2)/2
        const double Ws = W64 * k.sigma;
        for (int i = 0; i < 3; ++i) jp[i * ps] = rhoe * v64[i] + Ws * u64[i];
        jp[3 * ps] = a64 + pdd;                             // Z = tau~ + D + p
        jp[4 * ps] = pdd + ((rp[TAU * ps] + Dd) - a64);     // (E^2 + B^2)/2 = tau + D - a
    }
    if (!(pdd > 0.0) || !(gres * 1e9f <= gs) || !pconv || !isfinite(Ed[0] + Ed[1] + Ed[2] + W64))
        return ST_NEWTON;  // counted by the restart (stage_restarts)
    if constexpr (STATS) count_solve(k.hist, nit, pass + 1, 0);
    return ST_OK;
}

// One restart of the solve (starts 1 and 2 above): the same FP32 Newton phase
// and FP64 passes, from the ideal-limit E (START = 1) or along a continuation
// in a dt (START = 2). Used only after start 0 failed.
template <int NREF, bool STATS, int START>
__device__ __forceinline__ int stage_attempt(const double *rp, long long ps, double p_warm, const StageConst &k,
                                             double *qp, double *wp, double *jp = nullptr) {
    constexpr int start = START;
    const double gm1 = k.gamma - 1.0, gam = k.gamma;
    double tauB;
    float Bf[3], Sf[3], rEf[3], tauBf, Df, rhoef;
    {
        const double B[3] = {rp[BX * ps], rp[BY * ps], rp[BZ * ps]};
        const double Sv[3] = {rp[SX * ps], rp[SY * ps], rp[SZ * ps]};
        const double tau = rp[TAU * ps], Dd = rp[D * ps], rhoe = rp[RHOE * ps];
        tauB = tau - 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        for (int i = 0; i < 3; ++i) {
            const double rEi = rp[(EX + i) * ps];
            Bf[i] = f32_of(B[i]);
            Sf[i] = f32_of(Sv[i]);
            rEf[i] = f32_of(rEi);
            qp[(EX + i) * ps] = rEi;  // replaced by the root; left as r_E if the solve fails
        }
        tauBf = f32_of(tauB);
        Df = f32_of(Dd);
        rhoef = f32_of(rhoe);
        // source-free components equal r; psi and phi in closed form
        qp[D * ps] = Dd;
        qp[TAU * ps] = tau;
        qp[RHOE * ps] = rhoe;
        for (int i = 0; i < 3; ++i) {
            qp[(SX + i) * ps] = Sv[i];
            qp[(BX + i) * ps] = B[i];
        }
        qp[PSI * ps] = (rp[PSI * ps] + k.adt * rhoe) * k.cpsi;
        qp[PHI * ps] = rp[PHI * ps] * k.cpsi;
    }

    const float adtf = f32_of(k.adt), sigf = f32_of(k.sigma), gm1f = f32_of(gm1), gamf = f32_of(gam);
    const float scale = fmaxf(fmaxf(fabsf(rEf[0]), fabsf(rEf[1])), fmaxf(fabsf(rEf[2]), 1e-30f));
    int nit = 0, pass = 0;
    {
        // ---- FP32 Newton (start 2: a continuation of 7 levels in a dt)
        float E[3] = {rEf[0], rEf[1], rEf[2]};
        float p = f32_of(p_warm), dfdp = -1.f;
        float G[3], v[3], W, St[3], a, S2;
        float Minv[9], dpdE[3];
        bool have_jac = false, ok = true;
        if constexpr (start == 1) {  // the ideal-MHD limit E = -v x B, v recovered at E = r_E
            em_split(E, Sf, Bf, tauBf, Df, St, a, S2);
            if (!pres_solve_f32(p, a, S2, Df, gm1f, gamf, dfdp)) return ST_NEWTON;
            stage_resid(E, p, St, a, Bf, rEf, rhoef, adtf, sigf, G, v, W);
            cross(v, Bf, E);
            E[0] = -E[0]; E[1] = -E[1]; E[2] = -E[2];
        }
        constexpr int nlev = start == 2 ? 7 : 1;
        nit = 0;
        for (int lev = 0; lev < nlev && ok; ++lev) {
            // a dt 2^-(nlev-1-lev)
            const float adtl = nlev == 1 ? adtf : adtf * __int_as_float((127 - (nlev - 1 - lev)) << 23);
            em_split(E, Sf, Bf, tauBf, Df, St, a, S2);
            if (!pres_solve_f32(p, a, S2, Df, gm1f, gamf, dfdp)) {
                if (start == 0) return ST_C2P;  // r admits no primitives: no start can help
                ok = false;
                break;
            }
            stage_resid(E, p, St, a, Bf, rEf, rhoef, adtl, sigf, G, v, W);
            float gn = fmaxf(fmaxf(fabsf(G[0]), fabsf(G[1])), fabsf(G[2]));
            for (int it = 0; it < 24; ++it) {
                ++nit;
                // Jacobian columns dG/dE_k with duals; dp/dE_k by the implicit-function theorem
                float Jm[9];
                for (int kc = 0; kc < 3; ++kc) {
                    Dual<float> Ed[3] = {Dual<float>(E[0], kc == 0), Dual<float>(E[1], kc == 1),
                                         Dual<float>(E[2], kc == 2)};
                    Dual<float> Std[3], ad, S2d;
                    em_split(Ed, Sf, Bf, tauBf, Df, Std, ad, S2d);
                    Dual<float> pd(p);
                    Dual<float> fd = pres_resid(pd, ad, S2d, Df, gm1f, gamf);
                    pd = Dual<float>(p, -fd.d / dfdp);
                    dpdE[kc] = pd.d;
                    Dual<float> Gd[3], vd[3], Wd;
                    stage_resid(Ed, pd, Std, ad, Bf, rEf, rhoef, adtl, sigf, Gd, vd, Wd);
                    Jm[0 + kc] = Gd[0].d;
                    Jm[3 + kc] = Gd[1].d;
                    Jm[6 + kc] = Gd[2].d;
                }
                if (!inv3(Jm, Minv)) { ok = false; break; }
                have_jac = true;
                float dE[3];
                for (int i = 0; i < 3; ++i) dE[i] = Minv[3 * i] * G[0] + Minv[3 * i + 1] * G[1] + Minv[3 * i + 2] * G[2];
                float dn = fmaxf(fmaxf(fabsf(dE[0]), fabsf(dE[1])), fabsf(dE[2]));
                if (dn <= 2e-7f * fmaxf(scale, fmaxf(fmaxf(fabsf(E[0]), fabsf(E[1])), fabsf(E[2])))) break;
                // |G| at the FP32 noise floor (p and v carry ~2e-7 relative error):
                // further FP32 steps cannot improve E; the FP64 passes take over
                if (gn <= 1e-6f * resid_scale(E, rEf, v, Bf, W, rhoef, adtl, sigf)) break;
                // backtracking on |G|_inf; the shortest steps may raise |G| by at
                // most half (a way out of FP32 noise), never more
                float t = 1.f;
                bool accepted = false;
                for (int ls = 0; ls < 8; ++ls) {
                    float Et[3] = {E[0] - t * dE[0], E[1] - t * dE[1], E[2] - t * dE[2]};
                    float pt = p, dft = dfdp, Gt[3], vt[3], Wt, Stt[3], at, S2t;
                    em_split(Et, Sf, Bf, tauBf, Df, Stt, at, S2t);
                    if (pres_solve_f32(pt, at, S2t, Df, gm1f, gamf, dft)) {
                        stage_resid(Et, pt, Stt, at, Bf, rEf, rhoef, adtl, sigf, Gt, vt, Wt);
                        float gt = fmaxf(fmaxf(fabsf(Gt[0]), fabsf(Gt[1])), fabsf(Gt[2]));
                        if (gt < gn || (t < 0.02f && gt <= 1.5f * gn)) {
                            E[0] = Et[0]; E[1] = Et[1]; E[2] = Et[2];
                            p = pt; dfdp = dft; G[0] = Gt[0]; G[1] = Gt[1]; G[2] = Gt[2];
                            v[0] = vt[0]; v[1] = vt[1]; v[2] = vt[2]; W = Wt;
                            gn = gt;
                            accepted = true;
                            break;
                        }
                    }
                    t *= 0.5f;
                }
                if (!accepted) break;  // FP32 noise floor: hand over to the FP64 passes
            }
        }
        if (!ok || !have_jac) return ST_NEWTON;

        // ---- FP64 refinement passes. Pass k evaluates G in FP64 at E_k (one FP64
        // pressure step, started from a first-order prediction) and forms the
        // correction dE_k with the FP32 inverse Jacobian. The evaluation point at
        // which |G| reaches round-off of the magnitude of G's terms and the
        // pressure step is at FP64 round-off (at least the NREF-th) is the
        // result, with its own primitives (J amplifies any E/v mismatch by
        // sigma). Cells that need it take extra passes (up to 8).
        const float gs = resid_scale(E, rEf, v, Bf, W, rhoef, adtf, sigf);  // round-off scale of G
        // Acceptance |G| <= tol gs. The explicit stages evaluate J = sigma W (E + v x B
        // - (v.E) v) at the accepted E, which multiplies an E error by ~sigma dt W,
        // while G's own terms carry a dt sigma W: for stiff cells (a dt sigma W >> 1)
        // the tolerance shrinks by that factor, down to a few units of FP64
        // round-off of G's terms. Non-stiff cells keep 1e-12.
        const float itol = 1.f / fmaxf(1e-12f * s_rcp(1.f + adtf * sigf * W), 1e-15f);
        // FP64 inputs, read again (the stores above keep the compiler from reusing
        // the first loads' registers)
        const double B[3] = {rp[BX * ps], rp[BY * ps], rp[BZ * ps]};
        const double Sv[3] = {rp[SX * ps], rp[SY * ps], rp[SZ * ps]};
        const double rE[3] = {rp[EX * ps], rp[EY * ps], rp[EZ * ps]};
        const double Dd = rp[D * ps], rhoe = rp[RHOE * ps];
        const double tD = tauB + Dd, arho = k.adt * rhoe, asig = k.adt * k.sigma;
        double Ed[3] = {f64_of(E[0]), f64_of(E[1]), f64_of(E[2])};
        double pdd = f64_of(p);
        const double rdf = f64_of(1.f / dfdp);
        double St64[3], a64, S264, G64[3], v64[3], W64, u64[3];
        float gres = 0.f;
        bool pconv = false;
        for (pass = 0; pass < 8; ++pass) {  // constant trip count; the cap k.maxpass breaks below
            em_split_folded(Ed, Sv, B, tD, St64, a64, S264);
            const double dp = pres_resid(pdd, a64, S264, Dd, gm1, gam) * rdf;
            pdd -= dp;
            // the pressure step is at round-off: with the FP32 slope each step
            // gains ~7 digits, so the error left after this one is below 1e-13 p
            pconv = f32_of(fabs(dp)) <= 1e-6f * f32_of(pdd);
            stage_resid_folded(Ed, pdd, St64, a64, B, rE, arho, asig, G64, v64, W64, u64);
            float Gf[3] = {f32_of(G64[0]), f32_of(G64[1]), f32_of(G64[2])};
            // |G| in FP32 from the copy the correction uses (f32_of maps a NaN to an
            // infinity, so a non-finite G fails the tests)
            gres = fmaxf(fmaxf(fabsf(Gf[0]), fabsf(Gf[1])), fabsf(Gf[2]));
            if (pass >= NREF - 1 && gres * itol <= gs && pconv) break;
            float dE[3];
            for (int i = 0; i < 3; ++i) dE[i] = Minv[3 * i] * Gf[0] + Minv[3 * i + 1] * Gf[1] + Minv[3 * i + 2] * Gf[2];
            if (pass == 7 || pass == k.maxpass - 1) break;
            // first-order prediction of the pressure at the corrected E
            pdd -= f64_of(dpdE[0] * dE[0] + dpdE[1] * dE[1] + dpdE[2] * dE[2]);
            Ed[0] -= f64_of(dE[0]);
            Ed[1] -= f64_of(dE[1]);
            Ed[2] -= f64_of(dE[2]);
        }
        if (!(pdd > 0.0) || !(gres * 1e9f <= gs) || !pconv || !isfinite(Ed[0] + Ed[1] + Ed[2] + W64))
            return ST_NEWTON;
        wp[VX * ps] = v64[0];
        wp[VY * ps] = v64[1];
        wp[VZ * ps] = v64[2];
        wp[P * ps] = pdd;
        wp[LOR * ps] = W64;
        qp[EX * ps] = Ed[0];
        qp[EY * ps] = Ed[1];
        qp[EZ * ps] = Ed[2];
        if (jp) {
            const double Ws = W64 * k.sigma;
            for (int i = 0; i < 3; ++i) jp[i * ps] = rhoe * v64[i] + Ws * u64[i];
            jp[3 * ps] = a64 + pdd;
            jp[4 * ps] = pdd + ((rp[TAU * ps] + Dd) - a64);
        }
        if constexpr (STATS) count_solve(k.hist, nit, pass + 1, start);
        return ST_OK;
    }
}

// Starts 1 and 2 after start 0 failed. A solve that no start converges is
// counted as start 3.
template <int NREF, bool STATS>
__device__ int stage_restarts(const double *rp, long long ps, double p_warm, const StageConst &k, double *qp,
                              double *wp, int first = 1, double *jp = nullptr) {
    if (first <= 1 && stage_attempt<NREF, STATS, 1>(rp, ps, p_warm, k, qp, wp, jp) == ST_OK) return ST_OK;
    if (stage_attempt<NREF, STATS, 2>(rp, ps, p_warm, k, qp, wp, jp) == ST_OK) return ST_OK;
    if constexpr (STATS) count_solve(k.hist, 24, 8, 3);
    return ST_NEWTON;
}

// Primitive recovery of a conserved state (no source solve): FP32 root, then
// two FP64 Newton steps with the FP32 slope. Returns status; w = (v, p, W).
__device__ __forceinline__ int recover(const double q[NC], double p_warm, double gamma, double w[NW]) {
    const double gm1 = gamma - 1.0;
    const double B[3] = {q[BX], q[BY], q[BZ]}, E[3] = {q[EX], q[EY], q[EZ]}, Sv[3] = {q[SX], q[SY], q[SZ]};
    const double tauB = q[TAU] - 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    double St[3], a, S2;
    em_split(E, Sv, B, tauB, q[D], St, a, S2);
    float p = f32_of(p_warm), df = -1.f;
    if (!pres_solve_f32(p, f32_of(a), f32_of(S2), f32_of(q[D]), f32_of(gm1), f32_of(gamma), df)) return ST_C2P;
    double pd = f64_of(p), rdf = f64_of(1.f / df);
    pd -= pres_resid(pd, a, S2, q[D], gm1, gamma) * rdf;
    pd -= pres_resid(pd, a, S2, q[D], gm1, gamma) * rdf;
    double rZ = s_rcp(a + pd);
    w[VX] = St[0] * rZ;
    w[VY] = St[1] * rZ;
    w[VZ] = St[2] * rZ;
    w[P] = pd;
    w[LOR] = s_rsqrt(1.0 - (w[VX] * w[VX] + w[VY] * w[VY] + w[VZ] * w[VZ]));
    if (!(pd > 0.0) || !isfinite(w[LOR])) return ST_C2P;
    return ST_OK;
}

// Ohm's-law current J = varrho v + W sigma [E + v x B - (v.E) v] (FP64).
__device__ __forceinline__ void current(const double *q, const double *w, double sigma, double J[3]) {
    const double v[3] = {w[VX], w[VY], w[VZ]};
    const double B[3] = {q[BX], q[BY], q[BZ]}, E[3] = {q[EX], q[EY], q[EZ]};
    double vxB[3];
    cross(v, B, vxB);
    double vE = v[0] * E[0] + v[1] * E[1] + v[2] * E[2];
    double Ws = w[LOR] * sigma;
    for (int i = 0; i < 3; ++i) J[i] = q[RHOE] * v[i] + Ws * (E[i] + vxB[i] - vE * v[i]);
}

// Flux along direction `dir` (0 = x, 1 = y, 2 = z) of Eq. (resistive RMHD):
//   D v_d; Z v_i v_d + [p + (E^2+B^2)/2] delta_id - E_i E_d - B_i B_d; S_d - D v_d;
//   B: -eps_ijd E_j + delta_id phi; E: eps_ijd B_j + delta_id psi; J_d; E_d; B_d,
// with Z = rho h W^2 = tau - (E^2+B^2)/2 + D + p (no division needed).
// T is the flux arithmetic type; J is passed in (computed in FP64).
template <class T>
__device__ __forceinline__ void flux(const T q[NC], const T w[NW], const T J[3], int dir, T f[NC]) {
    const T E2B2 = q[EX] * q[EX] + q[EY] * q[EY] + q[EZ] * q[EZ] + q[BX] * q[BX] + q[BY] * q[BY] + q[BZ] * q[BZ];
    const T pem = w[P] + T(0.5) * E2B2;
    const T Z = (q[TAU] - T(0.5) * E2B2) + q[D] + w[P];
    // selects instead of indices computed from dir keep the arrays in registers
    const T vd = dir == 0 ? w[VX] : (dir == 1 ? w[VY] : w[VZ]);
    const T Ed = dir == 0 ? q[EX] : (dir == 1 ? q[EY] : q[EZ]), Bd = dir == 0 ? q[BX] : (dir == 1 ? q[BY] : q[BZ]);
    const T Zv = Z * vd;
    f[D] = q[D] * vd;
    f[SX] = Zv * w[VX] - q[EX] * Ed - q[BX] * Bd;
    f[SY] = Zv * w[VY] - q[EY] * Ed - q[BY] * Bd;
    f[SZ] = Zv * w[VZ] - q[EZ] * Ed - q[BZ] * Bd;
    if (dir == 0) f[SX] += pem; else if (dir == 1) f[SY] += pem; else f[SZ] += pem;
    f[TAU] = (dir == 0 ? q[SX] : (dir == 1 ? q[SY] : q[SZ])) - q[D] * vd;
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
    f[RHOE] = dir == 0 ? J[0] : (dir == 1 ? J[1] : J[2]);
    f[PSI] = Ed;
    f[PHI] = Bd;
}

} // namespace sf
} // namespace rmhd
