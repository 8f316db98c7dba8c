/*
 * rmhd_oracle.c -- plain FP64 CPU oracle for one SSP2(222) or SSP3(332) IMEX step of
 * resistive single-fluid and two-fluid special-relativistic MHD, written from
 * Wright & Hawke, "Resistive and multi-fluid RMHD on graphics processing
 * units" (arXiv:1808.09721).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library. It shares no code, header or constant
 * table with the CUDA library; it is slow on purpose and written so that each
 * function can be checked by eye against the equation it cites.
 *
 * What is computed (all FP64, built with -ffp-contract=off):
 *   - Sec. 2.1.1, Eq. (resistive RMHD) and Eq. (resistive prims): single-fluid
 *     conserved vector q = (D, S_i, tau, B^i, E^i, varrho, psi, phi), 14 vars,
 *     its flux along direction k and its source.
 *   - Sec. 2.1.2, Eq. (twoFluid cons) and Appendix A: two-fluid conserved
 *     vector q = (D, S_i, tau, Dbar, Sbar_i, taubar, B^i, E^i, psi, phi),
 *     18 vars, flux and source.
 *   - Sec. 2.1.3: primitive recovery. The EM part is removed from S and tau,
 *     then a one-unknown root in the pressure p (Newton with bisection
 *     safeguard) is iterated to a round-off fixed point. Two-fluid states are
 *     first split into species with the linear decomposition of Sec. 2.1.3.
 *   - Sec. 2.2.1, Eq. (implicit stage) and Tables 1-2: the SSP2(222) and
 *     SSP3(332) IMEX steps.
 *     Each implicit stage q = r + a*dt*Psi(q) is a per-cell root. Components
 *     with zero source are equal to r; psi and phi are linear; the remaining
 *     unknowns (E for one fluid; Sbar, taubar, E for two fluids) are found by
 *     Newton with a forward-difference Jacobian and a backtracking line search,
 *     iterated to a round-off fixed point.
 *   - Sec. 2.2.2: Lax-Friedrichs flux-vector splitting with alpha = 1 and
 *     componentwise WENO3 reconstruction (epsilon = 1e-6, power 2).
 *   - Boundary conditions: outflow (copy nearest interior cell) or periodic,
 *     two ghost cells per side.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Variable indices                                                     */
/* ------------------------------------------------------------------ */
/* single fluid, order of Eq. (resistive RMHD) */
enum { SF_D = 0, SF_S = 1, SF_TAU = 4, SF_B = 5, SF_E = 8, SF_RHOE = 11, SF_PSI = 12, SF_PHI = 13, SF_NC = 14 };
/* two fluids, order of Sec. 2.1.2 */
enum { TF_D = 0, TF_S = 1, TF_TAU = 4, TF_DB = 5, TF_SB = 6, TF_TAUB = 9, TF_B = 10, TF_E = 13, TF_PSI = 16, TF_PHI = 17, TF_NC = 18 };
/* user primitives: single fluid (rho, vx, vy, vz, p, Bx, By, Bz, Ex, Ey, Ez);
 * two fluids (rho_e, v_e, p_e, rho_p, v_p, p_p, B, E) with species 0 = e (mu_e), 1 = p (mu_p). */
enum { SF_NP = 11, TF_NP = 16 };
/* per-cell recovered primitives kept by the oracle: per species (rho, vx, vy, vz, p) */
enum { SF_NW = 5, TF_NW = 10 };

enum { ORC_OK = 0, ORC_ERR_C2P = -4, ORC_ERR_NEWTON = -3, ORC_ERR_INVALID = -1 };
enum { MODEL_SF = 0, MODEL_TF = 1 };
enum { BC_OUTFLOW = 0, BC_PERIODIC = 1 };

typedef struct {
    int model;
    int nx, ny;
    double xmin, xmax, ymin, ymax;
    double gamma, sigma, mu_e, mu_p, kappa;
    int bc_x, bc_y;
    int scheme;      /* 0: SSP2(222) (Table 1), 1: SSP3(332) (Table 2) */
    int nz;          /* cells along z (0 or 1: no z direction) */
    double zmin, zmax;
    int bc_z;
} orc_cfg;

/* Levi-Civita symbol on {0,1,2}. */
static double levi(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0.0;
    if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1)) return 1.0;
    return -1.0;
}

static void cross(const double a[3], const double b[3], double c[3])
{
    for (int i = 0; i < 3; i++) {
        c[i] = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) c[i] += levi(i, j, k) * a[j] * b[k];
    }
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* Primitive -> conserved (Eq. resistive prims, Eq. twoFluid cons)      */
/* ------------------------------------------------------------------ */

/* One species' hydrodynamic part: D = rho W, Stilde_i = rho h W^2 v_i,
 * tautilde = rho h W^2 - p - rho W, with W = 1/sqrt(1 - v^2) and
 * h = 1 + Gamma p / (rho (Gamma - 1)) (Sec. 2.1.1). */
static void hydro_p2c(double rho, const double v[3], double p, double gamma,
                      double *D, double St[3], double *taut)
{
    double W = 1.0 / sqrt(1.0 - dot(v, v));
    double h = 1.0 + gamma * p / (rho * (gamma - 1.0));
    double Z = rho * h * W * W;
    *D = rho * W;
    for (int i = 0; i < 3; i++) St[i] = Z * v[i];
    *taut = Z - p - rho * W;
}

/* Single fluid: prim = (rho, v, p, B, E); varrho, psi, phi given separately. */
int orc_sf_p2c(const double *prim, double varrho, double psi, double phi, double gamma, double *q)
{
    const double *v = prim + 1, *B = prim + 5, *E = prim + 8;
    double D, St[3], taut, ExB[3];
    if (!(prim[0] > 0.0) || !(prim[4] > 0.0) || !(dot(v, v) < 1.0)) return ORC_ERR_INVALID;
    hydro_p2c(prim[0], v, prim[4], gamma, &D, St, &taut);
    cross(E, B, ExB);
    q[SF_D] = D;
    for (int i = 0; i < 3; i++) q[SF_S + i] = St[i] + ExB[i];
    q[SF_TAU] = taut + 0.5 * (dot(E, E) + dot(B, B));
    for (int i = 0; i < 3; i++) { q[SF_B + i] = B[i]; q[SF_E + i] = E[i]; }
    q[SF_RHOE] = varrho;
    q[SF_PSI] = psi;
    q[SF_PHI] = phi;
    return ORC_OK;
}

/* Two fluids: prim = (rho_e, v_e, p_e, rho_p, v_p, p_p, B, E). Sums over
 * species of Eq. (twoFluid cons); the EM terms enter S and tau once. */
int orc_tf_p2c(const double *prim, double psi, double phi, double gamma, double mu_e, double mu_p, double *q)
{
    const double *B = prim + 10, *E = prim + 13;
    double mu[2] = { mu_e, mu_p }, ExB[3];
    for (int i = 0; i < TF_NC; i++) q[i] = 0.0;
    for (int s = 0; s < 2; s++) {
        const double *ps = prim + 5 * s;
        double D, St[3], taut;
        if (!(ps[0] > 0.0) || !(ps[4] > 0.0) || !(dot(ps + 1, ps + 1) < 1.0)) return ORC_ERR_INVALID;
        hydro_p2c(ps[0], ps + 1, ps[4], gamma, &D, St, &taut);
        q[TF_D] += D;
        q[TF_DB] += mu[s] * D;
        for (int i = 0; i < 3; i++) { q[TF_S + i] += St[i]; q[TF_SB + i] += mu[s] * St[i]; }
        q[TF_TAU] += taut;
        q[TF_TAUB] += mu[s] * taut;
    }
    cross(E, B, ExB);
    for (int i = 0; i < 3; i++) {
        q[TF_S + i] += ExB[i];
        q[TF_B + i] = B[i];
        q[TF_E + i] = E[i];
    }
    q[TF_TAU] += 0.5 * (dot(E, E) + dot(B, B));
    q[TF_PSI] = psi;
    q[TF_PHI] = phi;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Primitive recovery (Sec. 2.1.3)                                      */
/* ------------------------------------------------------------------ */

/* Residual of the pressure root for one species with hydrodynamic conserved
 * data (D, Stilde, tautilde). With Z = rho h W^2 = tautilde + D + p and
 * v = Stilde / Z, the Gamma-law EOS p = (Gamma - 1) rho eps holds exactly when
 *   f(p) = (Gamma - 1) [ Z (1 - v^2) - D sqrt(1 - v^2) ] - Gamma p = 0,
 * since Z (1 - v^2) = rho h = rho + Gamma p/(Gamma - 1) and D sqrt(1-v^2) = rho.
 * Returns f and its derivative df/dp. */
static void c2p_residual(double p, double D, double S2, double taut, double gamma, double *f, double *df)
{
    double Z = taut + D + p;
    double v2 = S2 / (Z * Z);
    double sq = sqrt(1.0 - v2); /* 1/W */
    *f = (gamma - 1.0) * (Z * (1.0 - v2) - D * sq) - gamma * p;
    /* d/dp [Z - S2/Z] = 1 + v2 ; d/dp [D sqrt(1 - S2/Z^2)] = D v2 / (Z sqrt(1-v2)) */
    *df = (gamma - 1.0) * (1.0 + v2 - D * v2 / (Z * sq)) - gamma;
}

/* Solve f(p) = 0 on the bracket (0, (Gamma-1)(tautilde + D)]: f(0) > 0 for a
 * physical state and f is decreasing for Gamma <= 2, so the root is unique.
 * Newton steps are kept inside the bracket by bisection; iteration stops at a
 * round-off fixed point (|dp| <= 4 ulp of p, or the bracket collapses).
 * out = (rho, vx, vy, vz, p). */
int orc_hydro_c2p(double D, const double St[3], double taut, double gamma, double *out)
{
    double S2 = dot(St, St);
    if (!(D > 0.0) || !(taut + D > sqrt(S2)) || !isfinite(S2) || !isfinite(taut)) return ORC_ERR_C2P;
    double lo = 0.0, hi = (gamma - 1.0) * (taut + D);
    double p = 0.5 * hi, f, df;
    int ok = 0;
    for (int it = 0; it < 200; it++) {
        c2p_residual(p, D, S2, taut, gamma, &f, &df);
        if (f == 0.0) { ok = 1; break; }
        if (f > 0.0) lo = p; else hi = p;
        double pn = p - f / df;
        if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
        if (fabs(pn - p) <= 4.0 * DBL_EPSILON * fabs(pn) || hi - lo <= 4.0 * DBL_EPSILON * hi) { p = pn; ok = 1; break; }
        p = pn;
    }
    if (!ok || !(p > 0.0)) return ORC_ERR_C2P;
    double Z = taut + D + p;
    double v[3] = { St[0] / Z, St[1] / Z, St[2] / Z };
    double W = 1.0 / sqrt(1.0 - dot(v, v));
    out[0] = D / W;
    out[1] = v[0]; out[2] = v[1]; out[3] = v[2];
    out[4] = p;
    return ORC_OK;
}

/* Single fluid: Stilde = S - E x B, tautilde = tau - (E^2 + B^2)/2, then the
 * hydrodynamic root. w = (rho, vx, vy, vz, p). */
int orc_sf_c2p(const double *q, double gamma, double *w)
{
    const double *B = q + SF_B, *E = q + SF_E;
    double ExB[3], St[3];
    cross(E, B, ExB);
    for (int i = 0; i < 3; i++) St[i] = q[SF_S + i] - ExB[i];
    double taut = q[SF_TAU] - 0.5 * (dot(E, E) + dot(B, B));
    return orc_hydro_c2p(q[SF_D], St, taut, gamma, w);
}

/* Two fluids: species split of Sec. 2.1.3,
 *   D_e = (Dbar - mu_p D)/(mu_e - mu_p),   D_p = (Dbar - mu_e D)/(mu_p - mu_e),
 * and the same linear split of (Stilde, Sbar) and (tautilde, taubar), where
 * Stilde = S - E x B and tautilde = tau - (E^2 + B^2)/2 are the species sums
 * of the hydrodynamic parts. w = (rho, v, p)_e, (rho, v, p)_p. */
int orc_tf_c2p(const double *q, double gamma, double mu_e, double mu_p, double *w)
{
    const double *B = q + TF_B, *E = q + TF_E;
    double ExB[3], St[3];
    cross(E, B, ExB);
    for (int i = 0; i < 3; i++) St[i] = q[TF_S + i] - ExB[i];
    double taut = q[TF_TAU] - 0.5 * (dot(E, E) + dot(B, B));
    double De = (q[TF_DB] - mu_p * q[TF_D]) / (mu_e - mu_p);
    double Dp = (q[TF_DB] - mu_e * q[TF_D]) / (mu_p - mu_e);
    double Se[3], Sp[3];
    for (int i = 0; i < 3; i++) {
        Se[i] = (q[TF_SB + i] - mu_p * St[i]) / (mu_e - mu_p);
        Sp[i] = (q[TF_SB + i] - mu_e * St[i]) / (mu_p - mu_e);
    }
    double te = (q[TF_TAUB] - mu_p * taut) / (mu_e - mu_p);
    double tp = (q[TF_TAUB] - mu_e * taut) / (mu_p - mu_e);
    int st = orc_hydro_c2p(De, Se, te, gamma, w);
    if (st) return st;
    return orc_hydro_c2p(Dp, Sp, tp, gamma, w + 5);
}

/* ------------------------------------------------------------------ */
/* Sources (Eq. resistive RMHD right-hand side; Appendix A)             */
/* ------------------------------------------------------------------ */

static double lorentz(const double v[3]) { return 1.0 / sqrt(1.0 - dot(v, v)); }

/* Ohm's law of Sec. 2.1.1: J_i = varrho v_i + W sigma [E_i + (v x B)_i - (v.E) v_i]. */
void orc_sf_current(const double *q, const double *w, double sigma, double *J)
{
    const double *v = w + 1, *B = q + SF_B, *E = q + SF_E;
    double W = lorentz(v), vxB[3];
    cross(v, B, vxB);
    double vE = dot(v, E);
    for (int i = 0; i < 3; i++)
        J[i] = q[SF_RHOE] * v[i] + W * sigma * (E[i] + vxB[i] - vE * v[i]);
}

/* Single fluid source: zero except E (-J), psi (varrho - kappa psi), phi (-kappa phi). */
void orc_sf_source(const double *q, const double *w, double sigma, double kappa, double *s)
{
    double J[3];
    for (int i = 0; i < SF_NC; i++) s[i] = 0.0;
    orc_sf_current(q, w, sigma, J);
    for (int i = 0; i < 3; i++) s[SF_E + i] = -J[i];
    s[SF_PSI] = q[SF_RHOE] - kappa * q[SF_PSI];
    s[SF_PHI] = -kappa * q[SF_PHI];
}

/* Two-fluid auxiliaries of Appendix A: varrho = sum mu_s rho_s W_s,
 * J = sum mu_s rho_s W_s v_s, omega_p^2 = sum mu_s^2 rho_s,
 * W = sum mu_s^2 rho_s W_s / omega_p^2, u = sum mu_s^2 rho_s W_s v_s / omega_p^2,
 * varrho_0 = W varrho - J.u. */
typedef struct { double varrho, J[3], wp2, W, u[3], varrho0; } tf_aux;

static void tf_auxiliaries(const double *w, double mu_e, double mu_p, tf_aux *a)
{
    double mu[2] = { mu_e, mu_p };
    memset(a, 0, sizeof(*a));
    for (int s = 0; s < 2; s++) {
        const double *ws = w + 5 * s;
        double Ws = lorentz(ws + 1);
        a->varrho += mu[s] * ws[0] * Ws;
        for (int i = 0; i < 3; i++) a->J[i] += mu[s] * ws[0] * Ws * ws[1 + i];
        a->wp2 += mu[s] * mu[s] * ws[0];
    }
    for (int s = 0; s < 2; s++) {
        const double *ws = w + 5 * s;
        double Ws = lorentz(ws + 1);
        a->W += mu[s] * mu[s] * ws[0] * Ws / a->wp2;
        for (int i = 0; i < 3; i++) a->u[i] += mu[s] * mu[s] * ws[0] * Ws * ws[1 + i] / a->wp2;
    }
    a->varrho0 = a->W * a->varrho - dot(a->J, a->u);
}

/* Two-fluid source of Appendix A, with eta = 1/sigma:
 *   Sbar_i: omega_p^2 [W E_i + (u x B)_i - eta (J_i - varrho u_i)]
 *   taubar: omega_p^2 [u.E - eta (varrho - varrho_0 W)]
 *   E: -J,  psi: varrho - kappa psi,  phi: -kappa phi. */
void orc_tf_source(const double *q, const double *w, double sigma, double kappa, double mu_e, double mu_p, double *s)
{
    tf_aux a;
    const double *B = q + TF_B, *E = q + TF_E;
    double eta = 1.0 / sigma, uxB[3];
    for (int i = 0; i < TF_NC; i++) s[i] = 0.0;
    tf_auxiliaries(w, mu_e, mu_p, &a);
    cross(a.u, B, uxB);
    for (int i = 0; i < 3; i++) {
        s[TF_SB + i] = a.wp2 * (a.W * E[i] + uxB[i] - eta * (a.J[i] - a.varrho * a.u[i]));
        s[TF_E + i] = -a.J[i];
    }
    s[TF_TAUB] = a.wp2 * (dot(a.u, E) - eta * (a.varrho - a.varrho0 * a.W));
    s[TF_PSI] = a.varrho - kappa * q[TF_PSI];
    s[TF_PHI] = -kappa * q[TF_PHI];
}

/* ------------------------------------------------------------------ */
/* Fluxes along direction k (Eq. resistive RMHD; Appendix A)             */
/* ------------------------------------------------------------------ */

/* Single fluid flux f^k:
 *   D v^k;  rho h W^2 v_i v_k + [p + (E^2+B^2)/2] delta_ik - E_i E_k - B_i B_k;
 *   S_k - D v^k;  -eps_ijk E_j + delta_ik phi;  eps_ijk B_j + delta_ik psi;
 *   J^k;  E^k;  B^k. */
void orc_sf_flux(const double *q, const double *w, double gamma, double sigma, int k, double *f)
{
    const double *v = w + 1, *B = q + SF_B, *E = q + SF_E;
    double rho = w[0], p = w[4];
    double W = lorentz(v);
    double h = 1.0 + gamma * p / (rho * (gamma - 1.0));
    double Z = rho * h * W * W, J[3];
    double pem = p + 0.5 * (dot(E, E) + dot(B, B));
    orc_sf_current(q, w, sigma, J);
    f[SF_D] = q[SF_D] * v[k];
    for (int i = 0; i < 3; i++)
        f[SF_S + i] = Z * v[i] * v[k] + (i == k ? pem : 0.0) - E[i] * E[k] - B[i] * B[k];
    f[SF_TAU] = q[SF_S + k] - q[SF_D] * v[k];
    for (int i = 0; i < 3; i++) {
        double fb = 0.0, fe = 0.0;
        for (int j = 0; j < 3; j++) { fb -= levi(i, j, k) * E[j]; fe += levi(i, j, k) * B[j]; }
        f[SF_B + i] = fb + (i == k ? q[SF_PHI] : 0.0);
        f[SF_E + i] = fe + (i == k ? q[SF_PSI] : 0.0);
    }
    f[SF_RHOE] = J[k];
    f[SF_PSI] = E[k];
    f[SF_PHI] = B[k];
}

/* Two-fluid flux f^j of Appendix A (species sums; EM stress counted once):
 *   D: sum rho_s W_s v_s^j
 *   S_i: sum (rho_s h_s W_s^2 v_si v_s^j + delta p_s) - E_i E^j - B_i B^j + delta (E^2+B^2)/2
 *   tau: S^j - sum D_s v_s^j
 *   Dbar: sum mu_s D_s v_s^j
 *   Sbar_i: sum mu_s (rho_s h_s W_s^2 v_si v_s^j + delta p_s)
 *   taubar: sum (taubar_s + mu_s p_s) v_s^j
 *   B_i: eps_ijk E_k + delta phi;  E_i: -eps_ijk B_k + delta psi;  psi: E^j;  phi: B^j. */
void orc_tf_flux(const double *q, const double *w, double gamma, double mu_e, double mu_p, int j, double *f)
{
    const double *B = q + TF_B, *E = q + TF_E;
    double mu[2] = { mu_e, mu_p };
    for (int i = 0; i < TF_NC; i++) f[i] = 0.0;
    double sumDv = 0.0;
    for (int s = 0; s < 2; s++) {
        const double *ws = w + 5 * s;
        double rho = ws[0], p = ws[4];
        const double *v = ws + 1;
        double W = lorentz(v);
        double h = 1.0 + gamma * p / (rho * (gamma - 1.0));
        double Z = rho * h * W * W;
        double Ds = rho * W;
        double taubar_s = mu[s] * (Z - p - rho * W);
        f[TF_D] += Ds * v[j];
        sumDv += Ds * v[j];
        f[TF_DB] += mu[s] * Ds * v[j];
        for (int i = 0; i < 3; i++) {
            double Sij = Z * v[i] * v[j] + (i == j ? p : 0.0);
            f[TF_S + i] += Sij;
            f[TF_SB + i] += mu[s] * Sij;
        }
        f[TF_TAUB] += (taubar_s + mu[s] * p) * v[j];
    }
    double em = 0.5 * (dot(E, E) + dot(B, B));
    for (int i = 0; i < 3; i++) f[TF_S + i] += -E[i] * E[j] - B[i] * B[j] + (i == j ? em : 0.0);
    f[TF_TAU] = q[TF_S + j] - sumDv;
    for (int i = 0; i < 3; i++) {
        double fb = 0.0, fe = 0.0;
        for (int k = 0; k < 3; k++) { fb += levi(i, j, k) * E[k]; fe -= levi(i, j, k) * B[k]; }
        f[TF_B + i] = fb + (i == j ? q[TF_PHI] : 0.0);
        f[TF_E + i] = fe + (i == j ? q[TF_PSI] : 0.0);
    }
    f[TF_PSI] = E[j];
    f[TF_PHI] = B[j];
}

/* ------------------------------------------------------------------ */
/* WENO3 (Sec. 2.2.2; Shu 1997, Jiang-Shu weights)                      */
/* ------------------------------------------------------------------ */

/* Face value at i+1/2 from the left-biased stencil (f_{i-1}, f_i, f_{i+1}):
 *   p0 = -f_{i-1}/2 + 3 f_i/2,  p1 = f_i/2 + f_{i+1}/2,
 *   beta0 = (f_i - f_{i-1})^2,  beta1 = (f_{i+1} - f_i)^2,
 *   alpha_k = d_k/(eps + beta_k)^2 with d = (1/3, 2/3), eps = 1e-6,
 *   value = (alpha0 p0 + alpha1 p1)/(alpha0 + alpha1).
 * The right-going face value of f^- is the mirror image: weno3(f_{i+2}, f_{i+1}, f_i). */
double orc_weno3(double fm, double f0, double fp)
{
    const double eps = 1e-6;
    double p0 = -0.5 * fm + 1.5 * f0;
    double p1 = 0.5 * f0 + 0.5 * fp;
    double b0 = (f0 - fm) * (f0 - fm);
    double b1 = (fp - f0) * (fp - f0);
    double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    return (a0 * p0 + a1 * p1) / (a0 + a1);
}

/* ------------------------------------------------------------------ */
/* Small dense linear solve (Gaussian elimination, partial pivoting)   */
/* ------------------------------------------------------------------ */
static int dense_solve(int n, double *A, double *b)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++) if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0 || !isfinite(A[piv * n + c])) return -1;
        if (piv != c) {
            for (int k = 0; k < n; k++) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double m = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= m * A[c * n + k];
            b[r] -= m * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Implicit stage (Eq. implicit stage with the diagonal coefficient a) */
/* ------------------------------------------------------------------ */

typedef struct {
    int model;
    const double *r;   /* explicit part of the stage, N_c values */
    double adt;        /* a_ii * dt */
    double gamma, sigma, kappa, mu_e, mu_p;
} stage_ctx;

static int nunk(int model) { return model == MODEL_SF ? 3 : 7; }

/* Build the full state q(x) from the unknowns x: components with zero source
 * keep their r value; psi = (r_psi + adt varrho)/(1 + adt kappa) and
 * phi = r_phi/(1 + adt kappa) solve their linear stage equations exactly. */
static void stage_assemble(const stage_ctx *c, const double *x, double *q)
{
    if (c->model == MODEL_SF) {
        memcpy(q, c->r, SF_NC * sizeof(double));
        for (int i = 0; i < 3; i++) q[SF_E + i] = x[i];
        q[SF_PSI] = (c->r[SF_PSI] + c->adt * c->r[SF_RHOE]) / (1.0 + c->adt * c->kappa);
        q[SF_PHI] = c->r[SF_PHI] / (1.0 + c->adt * c->kappa);
    } else {
        memcpy(q, c->r, TF_NC * sizeof(double));
        for (int i = 0; i < 3; i++) { q[TF_SB + i] = x[i]; q[TF_E + i] = x[4 + i]; }
        q[TF_TAUB] = x[3];
        /* varrho = Dbar for two fluids (charge density of Appendix A) */
        q[TF_PSI] = (c->r[TF_PSI] + c->adt * c->r[TF_DB]) / (1.0 + c->adt * c->kappa);
        q[TF_PHI] = c->r[TF_PHI] / (1.0 + c->adt * c->kappa);
    }
}

static void stage_unknowns(int model, const double *q, double *x)
{
    if (model == MODEL_SF) { for (int i = 0; i < 3; i++) x[i] = q[SF_E + i]; }
    else { for (int i = 0; i < 3; i++) { x[i] = q[TF_SB + i]; x[4 + i] = q[TF_E + i]; } x[3] = q[TF_TAUB]; }
}

/* G(x) = x - r_x - adt Psi_x(q(x)). Returns nonzero if the primitive
 * recovery of q(x) fails. */
static int stage_residual(const stage_ctx *c, const double *x, double *G, double *q, double *w)
{
    double s[TF_NC], rx[7];
    int n = nunk(c->model);
    stage_assemble(c, x, q);
    if (c->model == MODEL_SF) {
        if (orc_sf_c2p(q, c->gamma, w)) return -1;
        orc_sf_source(q, w, c->sigma, c->kappa, s);
    } else {
        if (orc_tf_c2p(q, c->gamma, c->mu_e, c->mu_p, w)) return -1;
        orc_tf_source(q, w, c->sigma, c->kappa, c->mu_e, c->mu_p, s);
    }
    double sx[7];
    stage_unknowns(c->model, s, sx);
    stage_unknowns(c->model, c->r, rx);
    for (int i = 0; i < n; i++) {
        G[i] = x[i] - rx[i] - c->adt * sx[i];
        if (!isfinite(G[i])) return -1;
    }
    return 0;
}

static double norm2sq(int n, const double *a) { double s = 0.0; for (int i = 0; i < n; i++) s += a[i] * a[i]; return s; }
static double norminf(int n, const double *a) { double s = 0.0; for (int i = 0; i < n; i++) if (fabs(a[i]) > s) s = fabs(a[i]); return s; }

/* Scale of round-off in the unknowns: max(|x|, |r_x|, |B|, |E|). x and r_x
 * enter G together; the field magnitude bounds the Ohm's-law terms of the E
 * rows (sigma W (E + v x B - (v.E) v), divided by the Jacobian ~ 1 + adt sigma W),
 * whose products can cancel to far below themselves when the root E ~ 0. */
static double stage_scale(const stage_ctx *c, int n, const double *x, const double *rs)
{
    const double *B = c->r + (c->model == MODEL_SF ? SF_B : TF_B);
    const double *E = x + (c->model == MODEL_SF ? 0 : 4);
    double sc = fmax(norminf(n, x), norminf(n, rs));
    sc = fmax(sc, fmax(norminf(3, B), norminf(3, E)));
    return fmax(sc, 1e-300);
}

/* Newton with forward-difference Jacobian and backtracking (Armijo 1e-4,
 * step halved down to 2^-10) from the start x; stops at a round-off fixed
 * point: the accepted step is at most 4 ulp of the round-off scale
 * (stage_scale), or the merit 1/2|G|^2 can no longer be decreased while the
 * Newton step is below 1e-10 of that scale (G has reached its round-off floor). */
static int newton_from(const stage_ctx *c, double *x, double *q, double *w, int *iters)
{
    int n = nunk(c->model);
    double G[7], Gt[7], xt[7], Jm[49], dx[7], qt[TF_NC], wt[TF_NW];
    if (stage_residual(c, x, G, q, w)) return -1;
    double xs = norminf(n, x);
    double rs[7];
    stage_unknowns(c->model, c->r, rs);
    if (norminf(n, rs) > xs) xs = norminf(n, rs);
    for (int it = 0; it < 60; it++) {
        if (iters) *iters = it;
        double m0 = 0.5 * norm2sq(n, G);
        if (m0 == 0.0) return 0;
        /* forward-difference Jacobian */
        for (int k = 0; k < n; k++) {
            double hk = 1.5e-8 * fmax(fabs(x[k]), fmax(xs, 1e-12));
            memcpy(xt, x, n * sizeof(double));
            xt[k] += hk;
            hk = xt[k] - x[k];
            if (stage_residual(c, xt, Gt, qt, wt)) {
                xt[k] = x[k] - hk;
                hk = xt[k] - x[k];
                if (stage_residual(c, xt, Gt, qt, wt)) return -1;
            }
            for (int i = 0; i < n; i++) Jm[i * n + k] = (Gt[i] - G[i]) / hk;
        }
        for (int i = 0; i < n; i++) dx[i] = -G[i];
        if (dense_solve(n, Jm, dx)) return -1;
        /* backtracking line search on 1/2 |G|^2 */
        double t = 1.0, m1 = 0.0;
        int accepted = 0;
        while (t >= 1.0 / 1024.0) {
            for (int i = 0; i < n; i++) xt[i] = x[i] + t * dx[i];
            if (!stage_residual(c, xt, Gt, qt, wt)) {
                m1 = 0.5 * norm2sq(n, Gt);
                if (m1 <= (1.0 - 2e-4 * t) * m0) { accepted = 1; break; }
            }
            t *= 0.5;
        }
        double scale = stage_scale(c, n, x, rs);
        double step = t * norminf(n, dx);
        if (!accepted) {
            /* No decrease of the merit: G is at its round-off floor. That is the
             * fixed point if the full Newton step is tiny; otherwise a stall. */
            return norminf(n, dx) <= 1e-10 * scale ? 0 : -1;
        }
        memcpy(x, xt, n * sizeof(double));
        memcpy(G, Gt, n * sizeof(double));
        memcpy(q, qt, (c->model == MODEL_SF ? SF_NC : TF_NC) * sizeof(double));
        memcpy(w, wt, (c->model == MODEL_SF ? SF_NW : TF_NW) * sizeof(double));
        if (step <= 4.0 * DBL_EPSILON * scale) return 0;
    }
    return -1;
}

/* Solve one implicit stage: q = r + adt Psi(q). Output q (N_c) and the
 * recovered primitives w (5 per species). Starts from x = r_x; if that fails
 * and the model is single fluid, restarts from the ideal-limit value
 * E = -v x B with v recovered from r. */
static int stage_solve(const stage_ctx *c, double *q, double *w)
{
    int n = nunk(c->model), it;
    double x[7];
    stage_unknowns(c->model, c->r, x);
    if (newton_from(c, x, q, w, &it) == 0) return ORC_OK;
    if (c->model == MODEL_SF) {
        double wr[SF_NW], vxB[3];
        if (orc_sf_c2p(c->r, c->gamma, wr) == 0) {
            cross(wr + 1, c->r + SF_B, vxB);
            for (int i = 0; i < 3; i++) x[i] = -vxB[i];
            if (newton_from(c, x, q, w, &it) == 0) return ORC_OK;
        }
    }
    /* continuation in a*dt: solve the stage for adt/2^m, ..., adt/2, adt, each
     * from the previous solution (the final root is the same; only the path differs) */
    for (int m = 3; m <= 12; m += 3) {
        stage_ctx cc = *c;
        int ok = 1;
        stage_unknowns(c->model, c->r, x);
        for (int k = m; k >= 0 && ok; k--) {
            cc.adt = ldexp(c->adt, -k);
            ok = newton_from(&cc, x, q, w, &it) == 0;
        }
        if (ok) return ORC_OK;
    }
    (void)n;
    return ORC_ERR_NEWTON;
}

int orc_sf_implicit(const double *r, double adt, double gamma, double sigma, double kappa, double *q, double *w)
{
    stage_ctx c = { MODEL_SF, r, adt, gamma, sigma, kappa, 0.0, 0.0 };
    return stage_solve(&c, q, w);
}

int orc_tf_implicit(const double *r, double adt, double gamma, double sigma, double kappa,
                    double mu_e, double mu_p, double *q, double *w)
{
    stage_ctx c = { MODEL_TF, r, adt, gamma, sigma, kappa, mu_e, mu_p };
    return stage_solve(&c, q, w);
}

/* ------------------------------------------------------------------ */
/* Grid, boundary conditions, flux divergence, IMEX steps              */
/* ------------------------------------------------------------------ */

typedef struct {
    orc_cfg cfg;
    int nc, nw, np;
    int nz;          /* cells along z (1: 1-D or 2-D grid) */
    int gx, gy, gz;  /* ghost layers: 2 in x; 2 in y (z) when ny (nz) > 1, else 0 */
    int NX, NY, NZ;  /* padded extents */
    int NR;          /* padded rows NY * NZ: arrays are [var][NZ][NY][NX] = [var][NR][NX] */
    double dx, dy, dz;
    double t;
    int fail_cell;   /* first failing interior cell (j*nx + i), -1 if none */
    double *q, *w;   /* state with ghosts: [var][NY][NX] */
    double *q1, *w1, *q2, *w2, *L1, *L2, *P1, *P2, *r;
    double *q3, *w3, *L3, *P3;  /* third stage of SSP3(332) */
} orc_sim;

static size_t cells(const orc_sim *s) { return (size_t)s->NX * s->NR; }
/* element (v, padded row R, padded column i); row R = k * NY + j */
static size_t at(const orc_sim *s, int v, int R, int i) { return ((size_t)v * s->NR + R) * s->NX + i; }
/* interior rows r = kk * ny + jj (the user layout [nz][ny][nx]) and their padded row */
static int nrows(const orc_sim *s) { return s->cfg.ny * s->nz; }
static int row_of(const orc_sim *s, int r) { return (r / s->cfg.ny + s->gz) * s->NY + r % s->cfg.ny + s->gy; }

/* Fill ghost cells of an array with nv variables. Outflow copies the nearest
 * interior cell; periodic wraps. x ghosts of the interior rows first, then y
 * ghost rows over the padded x extent, then z ghost planes over the padded
 * (y, x) extent, so edges and corners are consistent. */
static int ghost_src(int g, int n, int ng, int bc)
{
    /* padded index g (outside [ng, ng + n)) -> the padded interior index it copies */
    int lo = ng, hi = ng + n - 1;
    if (bc == BC_PERIODIC) {
        /* wrap modulo n: also for grids with fewer interior cells than ghost layers */
        int t = (g - ng) % n;
        return ng + (t < 0 ? t + n : t);
    }
    return g < lo ? lo : hi;
}

static void fill_ghosts(const orc_sim *s, double *a, int nv)
{
    int nx = s->cfg.nx, ny = s->cfg.ny, nz = s->nz, gx = s->gx, gy = s->gy, gz = s->gz;
    for (int v = 0; v < nv; v++) {
        for (int r = 0; r < nrows(s); r++) {
            int R = row_of(s, r);
            for (int g = 0; g < gx; g++) {
                int il = g, ir = gx + nx + g;
                a[at(s, v, R, il)] = a[at(s, v, R, ghost_src(il, nx, gx, s->cfg.bc_x))];
                a[at(s, v, R, ir)] = a[at(s, v, R, ghost_src(ir, nx, gx, s->cfg.bc_x))];
            }
        }
        for (int k = gz; k < gz + nz; k++)
            for (int g = 0; g < gy; g++) {
                int jl = g, jr = gy + ny + g;
                int sl = ghost_src(jl, ny, gy, s->cfg.bc_y), sr = ghost_src(jr, ny, gy, s->cfg.bc_y);
                for (int i = 0; i < s->NX; i++) {
                    a[at(s, v, k * s->NY + jl, i)] = a[at(s, v, k * s->NY + sl, i)];
                    a[at(s, v, k * s->NY + jr, i)] = a[at(s, v, k * s->NY + sr, i)];
                }
            }
        for (int g = 0; g < gz; g++) {
            int kl = g, kr = gz + nz + g;
            int sl = ghost_src(kl, nz, gz, s->cfg.bc_z), sr = ghost_src(kr, nz, gz, s->cfg.bc_z);
            for (int j = 0; j < s->NY; j++)
                for (int i = 0; i < s->NX; i++) {
                    a[at(s, v, kl * s->NY + j, i)] = a[at(s, v, sl * s->NY + j, i)];
                    a[at(s, v, kr * s->NY + j, i)] = a[at(s, v, sr * s->NY + j, i)];
                }
        }
    }
}

orc_sim *orc_create(const orc_cfg *cfg)
{
    if (cfg->nx < 1 || cfg->ny < 1) return NULL;
    if (cfg->model != MODEL_SF && cfg->model != MODEL_TF) return NULL;
    if (cfg->scheme != 0 && cfg->scheme != 1) return NULL;
    if (cfg->nz > 1 && cfg->ny < 2) return NULL;
    orc_sim *s = calloc(1, sizeof(orc_sim));
    s->cfg = *cfg;
    s->nc = cfg->model == MODEL_SF ? SF_NC : TF_NC;
    s->nw = cfg->model == MODEL_SF ? SF_NW : TF_NW;
    s->np = cfg->model == MODEL_SF ? SF_NP : TF_NP;
    s->nz = cfg->nz > 1 ? cfg->nz : 1;
    s->gx = 2;
    s->gy = cfg->ny > 1 ? 2 : 0;
    s->gz = s->nz > 1 ? 2 : 0;
    s->NX = cfg->nx + 2 * s->gx;
    s->NY = cfg->ny + 2 * s->gy;
    s->NZ = s->nz + 2 * s->gz;
    s->NR = s->NY * s->NZ;
    s->dx = (cfg->xmax - cfg->xmin) / cfg->nx;
    s->dy = (cfg->ymax - cfg->ymin) / cfg->ny;
    s->dz = s->nz > 1 ? (cfg->zmax - cfg->zmin) / s->nz : 1.0;
    s->fail_cell = -1;
    size_t nq = cells(s) * s->nc, nw = cells(s) * s->nw;
    s->q = calloc(nq, sizeof(double)); s->w = calloc(nw, sizeof(double));
    s->q1 = calloc(nq, sizeof(double)); s->w1 = calloc(nw, sizeof(double));
    s->q2 = calloc(nq, sizeof(double)); s->w2 = calloc(nw, sizeof(double));
    s->L1 = calloc(nq, sizeof(double)); s->L2 = calloc(nq, sizeof(double));
    s->P1 = calloc(nq, sizeof(double)); s->P2 = calloc(nq, sizeof(double));
    s->r = calloc(nq, sizeof(double));
    s->q3 = calloc(nq, sizeof(double)); s->w3 = calloc(nw, sizeof(double));
    s->L3 = calloc(nq, sizeof(double)); s->P3 = calloc(nq, sizeof(double));
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->q); free(s->w); free(s->q1); free(s->w1); free(s->q2); free(s->w2);
    free(s->L1); free(s->L2); free(s->P1); free(s->P2); free(s->r);
    free(s->q3); free(s->w3); free(s->L3); free(s->P3);
    free(s);
}

/* Gather/scatter one cell's variables from/to an SoA array. */
static void get_cell(const orc_sim *s, const double *a, int nv, int R, int i, double *c)
{ for (int v = 0; v < nv; v++) c[v] = a[at(s, v, R, i)]; }
static void put_cell(const orc_sim *s, double *a, int nv, int R, int i, const double *c)
{ for (int v = 0; v < nv; v++) a[at(s, v, R, i)] = c[v]; }

/* Set the initial state from user primitives [np][ny][nx] (interior cells).
 * psi = phi = 0 (Sec. 2.1.1). For one fluid the charge density is
 * initialised from Gauss's law varrho = div E with second-order central
 * differences, neighbours taken through the boundary conditions. */
int orc_set_prims(orc_sim *s, const double *prims)
{
    int nx = s->cfg.nx, ny = s->cfg.ny, np = s->np, nr = nrows(s);
    /* stage the user primitives in a ghosted array to take div E */
    double *P = calloc(cells(s) * np, sizeof(double));
    for (int v = 0; v < np; v++)
        for (int r = 0; r < nr; r++)
            for (int i = 0; i < nx; i++)
                P[at(s, v, row_of(s, r), i + s->gx)] = prims[((size_t)v * nr + r) * nx + i];
    fill_ghosts(s, P, np);
    int status = ORC_OK;
    for (int r = 0; r < nr && status == ORC_OK; r++) {
        int R = row_of(s, r);
        for (int i = s->gx; i < s->gx + nx; i++) {
            double pc[TF_NP], qc[TF_NC], wc[TF_NW];
            get_cell(s, P, np, R, i, pc);
            int st;
            if (s->cfg.model == MODEL_SF) {
                int ex = 8, ey = 9, ez = 10;
                double divE = (P[at(s, ex, R, i + 1)] - P[at(s, ex, R, i - 1)]) / (2.0 * s->dx);
                if (ny > 1) divE += (P[at(s, ey, R + 1, i)] - P[at(s, ey, R - 1, i)]) / (2.0 * s->dy);
                if (s->nz > 1) divE += (P[at(s, ez, R + s->NY, i)] - P[at(s, ez, R - s->NY, i)]) / (2.0 * s->dz);
                st = orc_sf_p2c(pc, divE, 0.0, 0.0, s->cfg.gamma, qc);
                memcpy(wc, pc, SF_NW * sizeof(double));
            } else {
                st = orc_tf_p2c(pc, 0.0, 0.0, s->cfg.gamma, s->cfg.mu_e, s->cfg.mu_p, qc);
                memcpy(wc, pc, TF_NW * sizeof(double));
            }
            if (st) { status = st; s->fail_cell = r * nx + (i - s->gx); break; }
            put_cell(s, s->q, s->nc, R, i, qc);
            put_cell(s, s->w, s->nw, R, i, wc);
        }
    }
    free(P);
    fill_ghosts(s, s->q, s->nc);
    fill_ghosts(s, s->w, s->nw);
    s->t = 0.0;
    return status;
}

/* Overwrite the conserved state (interior [nc][ny][nx]) and recover primitives. */
int orc_set_cons(orc_sim *s, const double *cons)
{
    int nx = s->cfg.nx, nr = nrows(s);
    for (int v = 0; v < s->nc; v++)
        for (int r = 0; r < nr; r++)
            for (int i = 0; i < nx; i++)
                s->q[at(s, v, row_of(s, r), i + s->gx)] = cons[((size_t)v * nr + r) * nx + i];
    fill_ghosts(s, s->q, s->nc);
    int status = ORC_OK;
    for (int r = 0; r < nr; r++)
        for (int i = s->gx; i < s->gx + nx; i++) {
            double qc[TF_NC], wc[TF_NW];
            int R = row_of(s, r);
            get_cell(s, s->q, s->nc, R, i, qc);
            int st = s->cfg.model == MODEL_SF ? orc_sf_c2p(qc, s->cfg.gamma, wc)
                                              : orc_tf_c2p(qc, s->cfg.gamma, s->cfg.mu_e, s->cfg.mu_p, wc);
            if (st && status == ORC_OK) { status = st; s->fail_cell = r * nx + (i - s->gx); }
            put_cell(s, s->w, s->nw, R, i, wc);
        }
    fill_ghosts(s, s->w, s->nw);
    return status;
}

static void copy_interior_out(const orc_sim *s, const double *a, int nv, double *out)
{
    int nx = s->cfg.nx, nr = nrows(s);
    for (int v = 0; v < nv; v++)
        for (int r = 0; r < nr; r++)
            for (int i = 0; i < nx; i++)
                out[((size_t)v * nr + r) * nx + i] = a[at(s, v, row_of(s, r), i + s->gx)];
}

int orc_get_cons(const orc_sim *s, double *out) { copy_interior_out(s, s->q, s->nc, out); return ORC_OK; }

/* Primitives in the user layout: one fluid (rho, v, p, B, E); two fluids
 * ((rho, v, p)_e, (rho, v, p)_p, B, E). */
int orc_get_prims(const orc_sim *s, double *out)
{
    int nx = s->cfg.nx, nr = nrows(s);
    size_t n = (size_t)nx * nr;
    copy_interior_out(s, s->w, s->nw, out);
    int b = s->cfg.model == MODEL_SF ? SF_B : TF_B;
    for (int c = 0; c < 6; c++)
        for (int r = 0; r < nr; r++)
            for (int i = 0; i < nx; i++)
                out[(s->nw + c) * n + (size_t)r * nx + i] = s->q[at(s, b + c, row_of(s, r), i + s->gx)];
    return ORC_OK;
}

/* The whole padded array (ghost cells included) of the conserved state
 * (which = 0, [nc][NZ][NY][NX]) or of the recovered primitives (which = 1,
 * [nw][NZ][NY][NX]); dims[3] receives (NX, NY, NZ). Exposes the ghost cells
 * that fill_ghosts wrote, for tests of the boundary conditions. */
int orc_get_padded(const orc_sim *s, int which, double *out, int *dims)
{
    const double *a = which == 0 ? s->q : s->w;
    int nv = which == 0 ? s->nc : s->nw;
    if (dims) { dims[0] = s->NX; dims[1] = s->NY; dims[2] = s->NZ; }
    if (out) memcpy(out, a, cells(s) * nv * sizeof(double));
    return ORC_OK;
}

double orc_time(const orc_sim *s) { return s->t; }
int orc_fail_cell(const orc_sim *s) { return s->fail_cell; }

static void cell_flux(const orc_sim *s, const double *qc, const double *wc, int k, double *f)
{
    if (s->cfg.model == MODEL_SF) orc_sf_flux(qc, wc, s->cfg.gamma, s->cfg.sigma, k, f);
    else orc_tf_flux(qc, wc, s->cfg.gamma, s->cfg.mu_e, s->cfg.mu_p, k, f);
}

/* L(q) = -sum_k (F_{k,+1/2} - F_{k,-1/2}) / dx_k with face fluxes
 * F = fhat^+ + fhat^-, f^{+-} = (f +- q)/2 (alpha = 1), fhat^+ from WENO3 on
 * (f^+_{i-1}, f^+_i, f^+_{i+1}) and fhat^- from WENO3 on (f^-_{i+2}, f^-_{i+1}, f^-_i).
 * q and w must have their ghost cells filled. Writes interior cells of L. */
void orc_flux_divergence(orc_sim *s, const double *q, const double *w, double *L)
{
    int nx = s->cfg.nx, ny = s->cfg.ny, nc = s->nc, nw = s->nw, nr = nrows(s);
    memset(L, 0, cells(s) * nc * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nr; r++) {
        int R = row_of(s, r);
        for (int i = s->gx; i < s->gx + nx; i++) {
            double Lc[TF_NC] = { 0 };
            for (int k = 0; k < 3; k++) {
                if ((k == 1 && ny < 2) || (k == 2 && s->nz < 2)) continue;
                /* neighbour steps along direction k: columns (x) or rows (y: 1, z: NY) */
                int di = k == 0 ? 1 : 0, dR = k == 0 ? 0 : (k == 1 ? 1 : s->NY);
                double dxk = k == 0 ? s->dx : (k == 1 ? s->dy : s->dz);
                /* fluxes at the four cells i-2..i+1 and i-1..i+2 */
                double fp[5][TF_NC], fm[5][TF_NC];
                for (int o = -2; o <= 2; o++) {
                    double qc[TF_NC], wc[TF_NW], f[TF_NC];
                    get_cell(s, q, nc, R + o * dR, i + o * di, qc);
                    get_cell(s, w, nw, R + o * dR, i + o * di, wc);
                    cell_flux(s, qc, wc, k, f);
                    for (int v = 0; v < nc; v++) {
                        fp[o + 2][v] = 0.5 * (f[v] + qc[v]);
                        fm[o + 2][v] = 0.5 * (f[v] - qc[v]);
                    }
                }
                for (int v = 0; v < nc; v++) {
                    /* face i+1/2 (offsets -1,0,1 for f^+; 2,1,0 for f^-) */
                    double Fr = orc_weno3(fp[1][v], fp[2][v], fp[3][v]) + orc_weno3(fm[4][v], fm[3][v], fm[2][v]);
                    /* face i-1/2 */
                    double Fl = orc_weno3(fp[0][v], fp[1][v], fp[2][v]) + orc_weno3(fm[3][v], fm[2][v], fm[1][v]);
                    Lc[v] -= (Fr - Fl) / dxk;
                }
            }
            for (int v = 0; v < nc; v++) L[at(s, v, R, i)] = Lc[v];
        }
    }
}

static void source_field(orc_sim *s, const double *q, const double *w, double *P)
{
    int nx = s->cfg.nx, nr = nrows(s);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; r++)
        for (int i = s->gx; i < s->gx + nx; i++) {
            double qc[TF_NC], wc[TF_NW], sc[TF_NC];
            int R = row_of(s, r);
            get_cell(s, q, s->nc, R, i, qc);
            get_cell(s, w, s->nw, R, i, wc);
            if (s->cfg.model == MODEL_SF) orc_sf_source(qc, wc, s->cfg.sigma, s->cfg.kappa, sc);
            else orc_tf_source(qc, wc, s->cfg.sigma, s->cfg.kappa, s->cfg.mu_e, s->cfg.mu_p, sc);
            put_cell(s, P, s->nc, R, i, sc);
        }
}

/* Solve the implicit stage q_out = r + adt Psi(q_out) on every interior cell. */
static int implicit_field(orc_sim *s, const double *r, double adt, double *qo, double *wo)
{
    int nx = s->cfg.nx, nr = nrows(s), status = ORC_OK, fail = -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int rr = 0; rr < nr; rr++)
        for (int i = s->gx; i < s->gx + nx; i++) {
            double rc[TF_NC], qc[TF_NC], wc[TF_NW];
            int R = row_of(s, rr), cell = rr * nx + (i - s->gx);
            get_cell(s, r, s->nc, R, i, rc);
            stage_ctx c = { s->cfg.model, rc, adt, s->cfg.gamma, s->cfg.sigma, s->cfg.kappa, s->cfg.mu_e, s->cfg.mu_p };
            int st = stage_solve(&c, qc, wc);
            if (st) {
#pragma omp critical
                { if (status == ORC_OK || cell < fail) { status = st; fail = cell; } }
            }
            put_cell(s, qo, s->nc, R, i, qc);
            put_cell(s, wo, s->nw, R, i, wc);
        }
    if (status) s->fail_cell = fail;
    return status;
}

/* Ghosts of the new state, then its primitives by recovery (Sec. 2.1.3). */
static int recover_state(orc_sim *s)
{
    int nc = s->nc, nx = s->cfg.nx, nr = nrows(s), status = ORC_OK;
    fill_ghosts(s, s->q, nc);
    for (int r = 0; r < nr; r++)
        for (int i = s->gx; i < s->gx + nx; i++) {
            double qc[TF_NC], wc[TF_NW];
            int R = row_of(s, r);
            get_cell(s, s->q, nc, R, i, qc);
            int c = s->cfg.model == MODEL_SF ? orc_sf_c2p(qc, s->cfg.gamma, wc)
                                             : orc_tf_c2p(qc, s->cfg.gamma, s->cfg.mu_e, s->cfg.mu_p, wc);
            if (c && status == ORC_OK) { status = ORC_ERR_C2P; s->fail_cell = r * nx + (i - s->gx); }
            put_cell(s, s->w, s->nw, R, i, wc);
        }
    fill_ghosts(s, s->w, s->nw);
    return status;
}

/* One SSP2(222) IMEX step (Table 1 with gamma = 1 - 1/sqrt(2)):
 *   q1 = q^n + g dt Psi(q1)
 *   q2 = q^n + dt L(q1) + (1 - 2g) dt Psi(q1) + g dt Psi(q2)
 *   q^{n+1} = q^n + dt/2 [L(q1) + L(q2)] + dt/2 [Psi(q1) + Psi(q2)]
 * Psi(q_j) is evaluated from (q_j, w_j). Ghost cells are refilled after each
 * stage; w^{n+1} comes from primitive recovery of q^{n+1}. */
int orc_ssp2_step(orc_sim *s, double dt)
{
    const double g = 1.0 - 1.0 / sqrt(2.0);
    int nc = s->nc, nx = s->cfg.nx;
    size_t n = cells(s) * nc;
    int st = implicit_field(s, s->q, g * dt, s->q1, s->w1);
    if (st) return st;
    fill_ghosts(s, s->q1, nc); fill_ghosts(s, s->w1, s->nw);
    source_field(s, s->q1, s->w1, s->P1);
    orc_flux_divergence(s, s->q1, s->w1, s->L1);
    for (size_t k = 0; k < n; k++) s->r[k] = s->q[k] + dt * s->L1[k] + (1.0 - 2.0 * g) * dt * s->P1[k];
    st = implicit_field(s, s->r, g * dt, s->q2, s->w2);
    if (st) return st;
    fill_ghosts(s, s->q2, nc); fill_ghosts(s, s->w2, s->nw);
    source_field(s, s->q2, s->w2, s->P2);
    orc_flux_divergence(s, s->q2, s->w2, s->L2);
    for (int v = 0; v < nc; v++)
        for (int rr = 0; rr < nrows(s); rr++)
            for (int i = s->gx; i < s->gx + nx; i++) {
                size_t k = at(s, v, row_of(s, rr), i);
                s->q[k] = s->q[k] + 0.5 * dt * (s->L1[k] + s->L2[k]) + 0.5 * dt * (s->P1[k] + s->P2[k]);
            }
    s->t += dt;
    return recover_state(s);
}

/* One SSP3(332) IMEX step (Table 2 with gamma = 1 - 1/sqrt(2)): explicit
 * tableau rows (0,0,0), (1,0,0), (1/4,1/4,0); implicit rows (g,0,0),
 * (1-2g,g,0), (1/2-g,0,g); weights (1/6,1/6,2/3) for both.
 *   q1 = q^n + g dt Psi(q1)
 *   q2 = q^n + dt L(q1) + dt [(1 - 2g) Psi(q1) + g Psi(q2)]
 *   q3 = q^n + dt [L(q1) + L(q2)]/4 + dt [(1/2 - g) Psi(q1) + g Psi(q3)]
 *   q^{n+1} = q^n + dt [L1/6 + L2/6 + 2 L3/3] + dt [Psi1/6 + Psi2/6 + 2 Psi3/3] */
int orc_ssp3_step(orc_sim *s, double dt)
{
    const double g = 1.0 - 1.0 / sqrt(2.0);
    int nc = s->nc, nx = s->cfg.nx;
    size_t n = cells(s) * nc;
    int st = implicit_field(s, s->q, g * dt, s->q1, s->w1);
    if (st) return st;
    fill_ghosts(s, s->q1, nc); fill_ghosts(s, s->w1, s->nw);
    source_field(s, s->q1, s->w1, s->P1);
    orc_flux_divergence(s, s->q1, s->w1, s->L1);
    for (size_t k = 0; k < n; k++) s->r[k] = s->q[k] + dt * s->L1[k] + (1.0 - 2.0 * g) * dt * s->P1[k];
    st = implicit_field(s, s->r, g * dt, s->q2, s->w2);
    if (st) return st;
    fill_ghosts(s, s->q2, nc); fill_ghosts(s, s->w2, s->nw);
    source_field(s, s->q2, s->w2, s->P2);
    orc_flux_divergence(s, s->q2, s->w2, s->L2);
    for (size_t k = 0; k < n; k++)
        s->r[k] = s->q[k] + 0.25 * dt * (s->L1[k] + s->L2[k]) + (0.5 - g) * dt * s->P1[k];
    st = implicit_field(s, s->r, g * dt, s->q3, s->w3);
    if (st) return st;
    fill_ghosts(s, s->q3, nc); fill_ghosts(s, s->w3, s->nw);
    source_field(s, s->q3, s->w3, s->P3);
    orc_flux_divergence(s, s->q3, s->w3, s->L3);
    for (int v = 0; v < nc; v++)
        for (int rr = 0; rr < nrows(s); rr++)
            for (int i = s->gx; i < s->gx + nx; i++) {
                size_t k = at(s, v, row_of(s, rr), i);
                s->q[k] = s->q[k] + dt * (s->L1[k] / 6.0 + s->L2[k] / 6.0 + 2.0 * s->L3[k] / 3.0) +
                          dt * (s->P1[k] / 6.0 + s->P2[k] / 6.0 + 2.0 * s->P3[k] / 3.0);
            }
    s->t += dt;
    return recover_state(s);
}

int orc_step(orc_sim *s, double dt, int nsteps)
{
    for (int k = 0; k < nsteps; k++) {
        int st = s->cfg.scheme == 1 ? orc_ssp3_step(s, dt) : orc_ssp2_step(s, dt);
        if (st) return st;
    }
    return ORC_OK;
}

/* L(q) of the current state (interior [nc][ny][nx]) -- exposes the flux
 * divergence for tests. */
int orc_current_L(orc_sim *s, double *out)
{
    orc_flux_divergence(s, s->q, s->w, s->L1);
    copy_interior_out(s, s->L1, s->nc, out);
    return ORC_OK;
}

/* Stage-1 implicit solve of the current state (q1 = q^n + a dt Psi(q1)),
 * returned as interior [nc][ny][nx]; leaves the state unchanged. */
int orc_stage_solve(orc_sim *s, double adt, double *qout, double *wout)
{
    int st = implicit_field(s, s->q, adt, s->q1, s->w1);
    copy_interior_out(s, s->q1, s->nc, qout);
    if (wout) copy_interior_out(s, s->w1, s->nw, wout);
    return st;
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
