// adjoint_sf.cuh -- reverse-mode (vector-Jacobian) products of the per-cell
// maps of the single-fluid model (Sec. 2.1.1 of Wright & Hawke,
// arXiv:1808.09721), used by the discrete adjoint of the SSP2(222) step.
//
// cell_vjp: given the adjoints of the cell's outputs -- its physical fluxes
// f_x, f_y (Eq. resistive RMHD, flux column) and the nonzero source entries
// Psi_E = -J, Psi_psi = varrho - kappa psi, Psi_phi = -kappa phi -- return the
// adjoint of its conserved state q and of sigma. The primitives are functions
// of q through the pressure root f(p; a, |S~|^2, D) = 0 of Sec. 2.1.3; their
// derivatives follow from the implicit-function theorem,
//   dp = -(f_a da + f_S2 dS2 + f_D dD) / f_p,
// so the reverse sweep needs only the converged pressure, not the iteration.
//
// p2c_vjp: adjoint of the primitive -> conserved map (Eq. resistive prims).
#pragma once
#include "physics_sf.cuh"

namespace rmhd {
namespace sf {

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Adjoints flowing in: fbar[dir][14] for dir < ndir (x, y, z; may be null when ndir = 0),
// sbar[5] for the source entries (E_x, E_y, E_z, psi, phi). Adds into qbar[14]
// and *sigbar. p is the converged pressure of q.
__device__ __forceinline__ void cell_vjp(const double q[NC], double p, double gamma, double sigma, double kappa,
                                         int ndir, const double fbar[3][NC], const double sbar[5], double qbar[NC],
                                         double *sigbar) {
    const double gm1 = gamma - 1.0;
    const double Dd = q[D], rho_e = q[RHOE];
    const double S[3] = {q[SX], q[SY], q[SZ]}, B[3] = {q[BX], q[BY], q[BZ]}, E[3] = {q[EX], q[EY], q[EZ]};
    // ---- forward recomputation
    double ExB[3];
    cross3(E, B, ExB);
    const double St[3] = {S[0] - ExB[0], S[1] - ExB[1], S[2] - ExB[2]};
    const double E2 = dot3(E, E), B2 = dot3(B, B);
    const double a = q[TAU] - 0.5 * (E2 + B2) + Dd;
    const double Z = a + p, rZ = s_rcp(Z);
    const double v[3] = {St[0] * rZ, St[1] * rZ, St[2] * rZ};
    const double v2 = dot3(v, v);
    const double W = s_rsqrt(1.0 - v2);
    double vxB[3];
    cross3(v, B, vxB);
    const double vE = dot3(v, E);
    const double u[3] = {E[0] + vxB[0] - vE * v[0], E[1] + vxB[1] - vE * v[1], E[2] + vxB[2] - vE * v[2]};

    // ---- reverse sweep
    double Db = 0, taub = 0, rhob = 0, psib = 0, phib = 0, pb = 0, Zb = 0, Wb = 0, pemb = 0;
    double Sb[3] = {0, 0, 0}, Bb[3] = {0, 0, 0}, Eb[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, Jb[3] = {0, 0, 0};
    // sources
    for (int i = 0; i < 3; ++i) Jb[i] -= sbar[i];
    rhob += sbar[3];
    psib -= kappa * sbar[3];
    phib -= kappa * sbar[4];
    // fluxes f_d: D v_d; Z v_i v_d + delta_id p_em - E_i E_d - B_i B_d; S_d - D v_d;
    // B: (phi, -E_z, E_y) / (E_z, phi, -E_x) / (-E_y, E_x, phi);
    // E: (psi, B_z, -B_y) / (-B_z, psi, B_x) / (B_y, -B_x, psi); J_d; E_d; B_d
    for (int d = 0; d < ndir; ++d) {
        const double *m = fbar[d];
        Db += (m[D] - m[TAU]) * v[d];
        vb[d] += (m[D] - m[TAU]) * Dd;
        for (int i = 0; i < 3; ++i) {
            const double ms = m[SX + i];
            Zb += ms * v[i] * v[d];
            vb[i] += ms * Z * v[d];
            vb[d] += ms * Z * v[i];
            Eb[i] -= ms * E[d];
            Eb[d] -= ms * E[i];
            Bb[i] -= ms * B[d];
            Bb[d] -= ms * B[i];
        }
        pemb += m[SX + d];
        Sb[d] += m[TAU];
        if (d == 0) {
            phib += m[BX]; Eb[2] -= m[BY]; Eb[1] += m[BZ];
            psib += m[EX]; Bb[2] += m[EY]; Bb[1] -= m[EZ];
        } else if (d == 1) {
            Eb[2] += m[BX]; phib += m[BY]; Eb[0] -= m[BZ];
            Bb[2] -= m[EX]; psib += m[EY]; Bb[0] += m[EZ];
        } else {
            Eb[1] -= m[BX]; Eb[0] += m[BY]; phib += m[BZ];
            Bb[1] += m[EX]; Bb[0] -= m[EY]; psib += m[EZ];
        }
        Jb[d] += m[RHOE];
        Eb[d] += m[PSI];
        Bb[d] += m[PHI];
    }
    // p_em = p + (E^2 + B^2)/2 ; the flux's Z = tau - (E^2+B^2)/2 + D + p is the same Z
    pb += pemb;
    for (int i = 0; i < 3; ++i) { Eb[i] += pemb * E[i]; Bb[i] += pemb * B[i]; }
    // J = varrho v + W sigma u,  u = E + v x B - (v.E) v
    const double Ju = dot3(Jb, u);
    rhob += dot3(Jb, v);
    for (int i = 0; i < 3; ++i) vb[i] += rho_e * Jb[i];
    Wb += sigma * Ju;
    *sigbar += W * Ju;
    double ub[3] = {W * sigma * Jb[0], W * sigma * Jb[1], W * sigma * Jb[2]};
    for (int i = 0; i < 3; ++i) Eb[i] += ub[i];
    double Bxu[3], uxv[3];
    cross3(B, ub, Bxu);
    cross3(ub, v, uxv);
    const double uv = dot3(ub, v);
    for (int i = 0; i < 3; ++i) {
        vb[i] += Bxu[i] - vE * ub[i] - uv * E[i];
        Bb[i] += uxv[i];
        Eb[i] -= uv * v[i];
    }
    // W = (1 - v^2)^(-1/2)
    const double W3 = W * W * W;
    for (int i = 0; i < 3; ++i) vb[i] += Wb * W3 * v[i];
    // v = S~ / Z
    const double vbv = dot3(vb, v);
    double Stb[3] = {vb[0] * rZ, vb[1] * rZ, vb[2] * rZ};
    Zb -= vbv * rZ;
    // Z = a + p
    double ab = Zb;
    pb += Zb;
    // pressure root (implicit-function theorem)
    const double fZ = gm1 * (1.0 + v2 - Dd * v2 * W * rZ);
    const double fp = fZ - gamma;
    const double fS2 = gm1 * (-rZ + 0.5 * Dd * W * rZ * rZ);
    const double fD = -gm1 / W;
    const double k = -pb * s_rcp(fp);
    ab += k * fZ;
    const double S2b = k * fS2;
    Db += k * fD;
    for (int i = 0; i < 3; ++i) Stb[i] += 2.0 * S2b * St[i];
    // a = tau - (E^2 + B^2)/2 + D
    taub += ab;
    Db += ab;
    for (int i = 0; i < 3; ++i) { Eb[i] -= ab * E[i]; Bb[i] -= ab * B[i]; }
    // S~ = S - E x B
    double BxS[3], SxE[3];
    cross3(B, Stb, BxS);
    cross3(Stb, E, SxE);
    for (int i = 0; i < 3; ++i) {
        Sb[i] += Stb[i];
        Eb[i] -= BxS[i];
        Bb[i] -= SxE[i];
    }
    qbar[D] += Db;
    qbar[TAU] += taub;
    qbar[RHOE] += rhob;
    qbar[PSI] += psib;
    qbar[PHI] += phib;
    for (int i = 0; i < 3; ++i) {
        qbar[SX + i] += Sb[i];
        qbar[BX + i] += Bb[i];
        qbar[EX + i] += Eb[i];
    }
}

// Adjoint of the primitive -> conserved map (Eq. resistive prims) of one cell
// with primitives (rho, v, p, B, E): qbar (D, S, tau, B, E entries) -> pbar[11].
// varrho, psi and phi are handled by the caller (Gauss's law; psi = phi = 0).
__device__ __forceinline__ void p2c_vjp(const double prim[11], double gamma, const double qbar[NC], double pbar[11]) {
    const double rho = prim[0], v[3] = {prim[1], prim[2], prim[3]}, p = prim[4];
    const double B[3] = {prim[5], prim[6], prim[7]}, E[3] = {prim[8], prim[9], prim[10]};
    const double W = 1.0 / sqrt(1.0 - dot3(v, v));
    const double rh = rho + gamma * p / (gamma - 1.0);  // rho h
    const double Zp = rh * W * W;
    const double Db = qbar[D], taub = qbar[TAU];
    const double Sb[3] = {qbar[SX], qbar[SY], qbar[SZ]};
    double rhob = 0, pb = 0, Wb = 0, vb[3], Bb[3], Eb[3];
    // D = rho W
    rhob += Db * W;
    Wb += Db * rho;
    // S = Zp v + E x B
    const double Zpb = dot3(Sb, v) + taub;
    for (int i = 0; i < 3; ++i) vb[i] = Zp * Sb[i];
    double BxS[3], SxE[3];
    cross3(B, Sb, BxS);
    cross3(Sb, E, SxE);
    for (int i = 0; i < 3; ++i) { Eb[i] = BxS[i] + taub * E[i] + qbar[EX + i]; Bb[i] = SxE[i] + taub * B[i] + qbar[BX + i]; }
    // tau = Zp - p + (E^2 + B^2)/2 - rho W
    pb -= taub;
    rhob -= taub * W;
    Wb -= taub * rho;
    // Zp = (rho + Gamma p / (Gamma - 1)) W^2
    rhob += Zpb * W * W;
    pb += Zpb * gamma / (gamma - 1.0) * W * W;
    Wb += Zpb * 2.0 * rh * W;
    // W = (1 - v^2)^(-1/2)
    const double W3 = W * W * W;
    for (int i = 0; i < 3; ++i) vb[i] += Wb * W3 * v[i];
    pbar[0] = rhob;
    pbar[1] = vb[0];
    pbar[2] = vb[1];
    pbar[3] = vb[2];
    pbar[4] = pb;
    for (int i = 0; i < 3; ++i) { pbar[5 + i] = Bb[i]; pbar[8 + i] = Eb[i]; }
}

} // namespace sf
} // namespace rmhd
