// adjoint_tf.cuh -- reverse-mode (vector-Jacobian) products of the per-cell
// maps of the two-fluid model (Sec. 2.1.2, Sec. 2.1.3 and Appendix A of Wright
// & Hawke, arXiv:1808.09721), used by the discrete adjoint of the IMEX step.
//
// cell_vjp: given the adjoints of the cell's outputs -- its physical fluxes
// f_x, f_y, f_z (Appendix A, flux column) and the nonzero source entries
// (Sbar, taubar, E, psi, phi) -- return the adjoint of its conserved state q
// and of sigma (eta = 1/sigma in the Sbar and taubar sources). The primitives
// (v_s, p_s, Z_s = rho_s h_s W_s^2 of each species) are functions of q through
// the linear species split of Sec. 2.1.3 and one pressure root per species;
// the root's derivative follows from the implicit-function theorem, so the
// reverse sweep needs only the converged pressures.
//
// p2c_vjp: adjoint of the primitive -> conserved map (Eq. twoFluid cons).
#pragma once
#include "physics_tf.cuh"
#include "adjoint_sf.cuh"

namespace rmhd {
namespace tf {

using sf::cross3;
using sf::dot3;

// Adjoints flowing in: fbar[dir][18] for dir < ndir (may be zero-filled when
// ndir = 0), sbar[9] = (Sbar_x, Sbar_y, Sbar_z, taubar, E_x, E_y, E_z, psi,
// phi) for the source entries. w: the cell's primitives (v, p, Z per species,
// electrons first). Adds into qbar[18] and *sigbar.
__device__ __forceinline__ void cell_vjp(const double q[NC], const double w[NW], const Phys &ph, int ndir,
                                         const double fbar[3][NC], const double sbar[9], double qbar[NC],
                                         double *sigbar) {
    const double gm1 = ph.gamma - 1.0, gam = ph.gamma;
    const double mu[2] = {ph.mu_e, ph.mu_p};
    const double cbar[2] = {ph.inv_dmu, -ph.inv_dmu}, ctot[2] = {-ph.mu_p * ph.inv_dmu, ph.mu_e * ph.inv_dmu};
    const double B[3] = {q[BX], q[BY], q[BZ]}, E[3] = {q[EX], q[EY], q[EZ]};
    // ---- forward recomputation: species split and per-species primitives
    double Ds[2], Sts[2][3], v[2][3], Zs[2], ps[2], sq[2], W[2];
    double ExB[3];
    cross3(E, B, ExB);
    const double St[3] = {q[SX] - ExB[0], q[SY] - ExB[1], q[SZ] - ExB[2]};
    for (int s = 0; s < 2; ++s) {
        Ds[s] = cbar[s] * q[DB] + ctot[s] * q[D];
        for (int i = 0; i < 3; ++i) {
            Sts[s][i] = cbar[s] * q[SBX + i] + ctot[s] * St[i];
            v[s][i] = w[5 * s + VX + i];
        }
        ps[s] = w[5 * s + P];
        Zs[s] = w[5 * s + ZZ];
        const double om = 1.0 - dot3(v[s], v[s]);
        sq[s] = om * s_rsqrt(om);
        W[s] = s_rsqrt(om);
    }
    // aggregates of the sources (physics_tf.cuh: source_terms)
    double M0 = 0.0, wp2 = 0.0, vr = 0.0, M1[3] = {0, 0, 0}, J[3] = {0, 0, 0};
    for (int s = 0; s < 2; ++s) {
        M0 += mu[s] * mu[s] * Ds[s];
        wp2 += mu[s] * mu[s] * Ds[s] * sq[s];
        vr += mu[s] * Ds[s];
        for (int i = 0; i < 3; ++i) {
            M1[i] += mu[s] * mu[s] * Ds[s] * v[s][i];
            J[i] += mu[s] * Ds[s] * v[s][i];
        }
    }
    const double eta = ph.eta;
    const double JM1 = dot3(J, M1), num = M0 * vr - JM1, rwp = s_rcp(wp2), r0 = num * rwp;
    const double Tq = wp2 * vr - M0 * r0;
    const double U[3] = {wp2 * J[0] - vr * M1[0], wp2 * J[1] - vr * M1[1], wp2 * J[2] - vr * M1[2]};

    // ---- reverse sweep
    double Dsb[2] = {0, 0}, vb[2][3] = {{0, 0, 0}, {0, 0, 0}}, pb[2] = {0, 0}, Zb[2] = {0, 0}, sqb[2] = {0, 0};
    double Eb[3] = {0, 0, 0}, Bb[3] = {0, 0, 0}, Sqb[3] = {0, 0, 0};
    double Db = 0.0, DBb = 0.0, taub = 0.0, psib = 0.0, phib = 0.0, etab = 0.0;
    // sources: Sbar = M0 E + M1 x B - eta U, taubar = M1.E - eta T, E = -J,
    // psi = varrho - kappa psi, phi = -kappa phi
    double M0b = 0.0, wp2b = 0.0, vrb = 0.0, M1b[3] = {0, 0, 0}, Jb[3] = {0, 0, 0};
    {
        const double SBb[3] = {sbar[0], sbar[1], sbar[2]}, TBb = sbar[3];
        for (int i = 0; i < 3; ++i) Jb[i] -= sbar[4 + i];
        vrb += sbar[7];
        psib -= ph.kappa * sbar[7];
        phib -= ph.kappa * sbar[8];
        // taubar
        for (int i = 0; i < 3; ++i) { M1b[i] += TBb * E[i]; Eb[i] += TBb * M1[i]; }
        const double Tb = -eta * TBb;
        etab -= TBb * Tq;
        wp2b += Tb * vr;
        vrb += Tb * wp2;
        M0b -= Tb * r0;
        const double r0b = -Tb * M0;
        const double numb = r0b * rwp;
        wp2b -= r0b * r0 * rwp;
        M0b += numb * vr;
        vrb += numb * M0;
        for (int i = 0; i < 3; ++i) { Jb[i] -= numb * M1[i]; M1b[i] -= numb * J[i]; }
        // Sbar
        M0b += dot3(SBb, E);
        for (int i = 0; i < 3; ++i) Eb[i] += M0 * SBb[i];
        double BxS[3], SxM[3];
        cross3(B, SBb, BxS);
        cross3(SBb, M1, SxM);
        for (int i = 0; i < 3; ++i) { M1b[i] += BxS[i]; Bb[i] += SxM[i]; }
        etab -= dot3(SBb, U);
        const double Ub[3] = {-eta * SBb[0], -eta * SBb[1], -eta * SBb[2]};
        wp2b += dot3(Ub, J);
        vrb -= dot3(Ub, M1);
        for (int i = 0; i < 3; ++i) { Jb[i] += wp2 * Ub[i]; M1b[i] -= vr * Ub[i]; }
    }
    // aggregates -> species
    for (int s = 0; s < 2; ++s) {
        const double m2 = mu[s] * mu[s];
        Dsb[s] += m2 * M0b + m2 * sq[s] * wp2b + mu[s] * vrb + m2 * dot3(M1b, v[s]) + mu[s] * dot3(Jb, v[s]);
        sqb[s] += m2 * Ds[s] * wp2b;
        for (int i = 0; i < 3; ++i) vb[s][i] += m2 * Ds[s] * M1b[i] + mu[s] * Ds[s] * Jb[i];
    }
    // fluxes along d (physics_tf.cuh: flux)
    for (int d = 0; d < ndir; ++d) {
        const double *m = fbar[d];
        const double mD = m[D] - m[TAU];  // tau^d = S_d - D^d
        Sqb[d] += m[TAU];
        for (int s = 0; s < 2; ++s) {
            const double vd = v[s][d];
            Dsb[s] += (mD + mu[s] * m[DB] - mu[s] * m[TAUB]) * vd;
            vb[s][d] += (mD + mu[s] * m[DB]) * Ds[s] + mu[s] * m[TAUB] * (Zs[s] - Ds[s]);
            Zb[s] += mu[s] * m[TAUB] * vd;
            for (int i = 0; i < 3; ++i) {
                const double ms = m[SX + i] + mu[s] * m[SBX + i];
                Zb[s] += ms * vd * v[s][i];
                vb[s][d] += ms * Zs[s] * v[s][i];
                vb[s][i] += ms * Zs[s] * vd;
            }
            pb[s] += m[SX + d] + mu[s] * m[SBX + d];
        }
        for (int i = 0; i < 3; ++i) {
            const double ms = m[SX + i];
            Eb[i] -= ms * E[d];
            Eb[d] -= ms * E[i];
            Bb[i] -= ms * B[d];
            Bb[d] -= ms * B[i];
            Eb[i] += m[SX + d] * E[i];  // delta_id (E^2 + B^2)/2
            Bb[i] += m[SX + d] * B[i];
        }
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
        Eb[d] += m[PSI];
        Bb[d] += m[PHI];
    }
    // per-species recovery: v = S~_s / Z, Z = a + p, p the root of
    // f(p; a, |S~_s|^2, D_s) = 0 (implicit-function theorem), a = tau~_s + D_s
    double Stsb[2][3], ttsb[2];
    for (int s = 0; s < 2; ++s) {
        for (int i = 0; i < 3; ++i) vb[s][i] -= sqb[s] * v[s][i] / sq[s];  // sq = sqrt(1 - v^2)
        const double rZ = s_rcp(Zs[s]);
        const double vbv = dot3(vb[s], v[s]);
        for (int i = 0; i < 3; ++i) Stsb[s][i] = vb[s][i] * rZ;
        Zb[s] -= vbv * rZ;
        double ab = Zb[s];
        double pbt = pb[s] + Zb[s];
        const double v2 = dot3(v[s], v[s]);
        const double fZ = gm1 * (1.0 + v2 - Ds[s] * v2 * W[s] * rZ);
        const double fp = fZ - gam;
        const double fS2 = gm1 * (-rZ + 0.5 * Ds[s] * W[s] * rZ * rZ);
        const double fD = -gm1 * sq[s];
        const double k = -pbt * s_rcp(fp);
        ab += k * fZ;
        const double S2b = k * fS2;
        Dsb[s] += k * fD;
        for (int i = 0; i < 3; ++i) Stsb[s][i] += 2.0 * S2b * Sts[s][i];
        ttsb[s] = ab;
        Dsb[s] += ab;
    }
    (void)ps;
    // species split of (D, Dbar), (S~, Sbar), (tau~, taubar)
    double Stb[3] = {0, 0, 0}, tautb = 0.0, SBqb[3] = {0, 0, 0}, TBqb = 0.0;
    for (int s = 0; s < 2; ++s) {
        DBb += cbar[s] * Dsb[s];
        Db += ctot[s] * Dsb[s];
        for (int i = 0; i < 3; ++i) {
            SBqb[i] += cbar[s] * Stsb[s][i];
            Stb[i] += ctot[s] * Stsb[s][i];
        }
        TBqb += cbar[s] * ttsb[s];
        tautb += ctot[s] * ttsb[s];
    }
    // S~ = S - E x B, tau~ = tau - (E^2 + B^2)/2
    double BxS[3], SxE[3];
    cross3(B, Stb, BxS);
    cross3(Stb, E, SxE);
    for (int i = 0; i < 3; ++i) {
        Sqb[i] += Stb[i];
        Eb[i] -= BxS[i] + tautb * E[i];
        Bb[i] -= SxE[i] + tautb * B[i];
    }
    taub += tautb;
    qbar[D] += Db;
    qbar[TAU] += taub;
    qbar[DB] += DBb;
    qbar[TAUB] += TBqb;
    qbar[PSI] += psib;
    qbar[PHI] += phib;
    for (int i = 0; i < 3; ++i) {
        qbar[SX + i] += Sqb[i];
        qbar[SBX + i] += SBqb[i];
        qbar[BX + i] += Bb[i];
        qbar[EX + i] += Eb[i];
    }
    // eta = 1 / sigma
    *sigbar -= etab * eta * eta;
}

// Adjoint of the primitive -> conserved map (Eq. twoFluid cons) of one cell
// with primitives (rho_e, v_e, p_e, rho_p, v_p, p_p, B, E): qbar[18] ->
// pbar[16]. psi = phi = 0 are constants.
__device__ __forceinline__ void p2c_vjp(const double prim[16], const Phys &ph, const double qbar[NC],
                                        double pbar[16]) {
    const double gamma = ph.gamma, mu[2] = {ph.mu_e, ph.mu_p};
    const double B[3] = {prim[10], prim[11], prim[12]}, E[3] = {prim[13], prim[14], prim[15]};
    for (int s = 0; s < 2; ++s) {
        const double *pr = prim + 5 * s;
        const double rho = pr[0], v[3] = {pr[1], pr[2], pr[3]}, p = pr[4];
        const double W = 1.0 / sqrt(1.0 - dot3(v, v));
        const double rh = rho + gamma * p / (gamma - 1.0);
        const double Zp = rh * W * W;
        // this species' hydrodynamic parts enter the totals and the mu-weighted sums
        const double Dsb = qbar[D] + mu[s] * qbar[DB], tsb = qbar[TAU] + mu[s] * qbar[TAUB];
        const double Ssb[3] = {qbar[SX] + mu[s] * qbar[SBX], qbar[SY] + mu[s] * qbar[SBY],
                               qbar[SZ] + mu[s] * qbar[SBZ]};
        double rhob = 0, pb = 0, Wb = 0, vb[3];
        rhob += Dsb * W;
        Wb += Dsb * rho;
        const double Zpb = dot3(Ssb, v) + tsb;
        for (int i = 0; i < 3; ++i) vb[i] = Zp * Ssb[i];
        pb -= tsb;
        rhob -= tsb * W;
        Wb -= tsb * rho;
        rhob += Zpb * W * W;
        pb += Zpb * gamma / (gamma - 1.0) * W * W;
        Wb += Zpb * 2.0 * rh * W;
        const double W3 = W * W * W;
        for (int i = 0; i < 3; ++i) vb[i] += Wb * W3 * v[i];
        pbar[5 * s] = rhob;
        for (int i = 0; i < 3; ++i) pbar[5 * s + 1 + i] = vb[i];
        pbar[5 * s + 4] = pb;
    }
    const double Sb[3] = {qbar[SX], qbar[SY], qbar[SZ]}, taub = qbar[TAU];
    double BxS[3], SxE[3];
    cross3(B, Sb, BxS);
    cross3(Sb, E, SxE);
    for (int i = 0; i < 3; ++i) {
        pbar[13 + i] = BxS[i] + taub * E[i] + qbar[EX + i];
        pbar[10 + i] = SxE[i] + taub * B[i] + qbar[BX + i];
    }
}

} // namespace tf
} // namespace rmhd
