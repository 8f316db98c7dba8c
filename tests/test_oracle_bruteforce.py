"""Brute-force pin of the oracle's implicit stage (no GPU).

The paper solves each implicit stage as a root of the full N_c-dimensional
system q = r + a dt Psi(q) (Eq. implicit stage; Sec. 2.2.1 uses CMINPACK on
all N_c components). The oracle instead solves a reduced system (only the
components with a nonzero source are unknowns, psi and phi in closed form).
Here a 40-digit mpmath solve of the full system -- mpmath's own multi-
dimensional Newton and bracketing root finder, with the model written from
the printed definitions -- must agree with the oracle to 1e-12. Tiny inputs:
a handful of cells.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_09721_gb300 import workloads as WL

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp
G = 1.0 - 1.0 / math.sqrt(2.0)


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _hydro_prims(D, St, taut, gamma):
    """Root of the Gamma-law EOS written with the textbook quantities:
    v = St/(taut + D + p), W, rho = D/W, h = (taut + D + p)/(rho W^2),
    eps = h - 1 - p/rho, residual (Gamma - 1) rho eps - p (Sec. 2.1.3)."""
    S2 = _dot(St, St)

    def f(p):
        Z = taut + D + p
        v2 = S2 / Z ** 2
        W = 1 / mp.sqrt(1 - v2)
        rho = D / W
        h = Z / (rho * W ** 2)
        eps = h - 1 - p / rho
        return (gamma - 1) * rho * eps - p

    lo = mp.mpf(10) ** -30
    hi = 2 * (taut + D) + 1
    p = mp.findroot(f, (lo, hi), solver="anderson")
    Z = taut + D + p
    v = [s / Z for s in St]
    W = 1 / mp.sqrt(1 - _dot(v, v))
    return D / W, v, p, W


def _sf_source_full(q, gamma, sigma, kappa):
    D, S, tau, B, E, varrho, psi, phi = q[0], q[1:4], q[4], q[5:8], q[8:11], q[11], q[12], q[13]
    ExB = _cross(E, B)
    St = [S[i] - ExB[i] for i in range(3)]
    taut = tau - (_dot(E, E) + _dot(B, B)) / 2
    rho, v, p, W = _hydro_prims(D, St, taut, gamma)
    vxB = _cross(v, B)
    vE = _dot(v, E)
    J = [varrho * v[i] + W * sigma * (E[i] + vxB[i] - vE * v[i]) for i in range(3)]
    s = [mp.mpf(0)] * 14
    for i in range(3):
        s[8 + i] = -J[i]
    s[12] = varrho - kappa * psi
    s[13] = -kappa * phi
    return s


def _tf_source_full(q, gamma, sigma, kappa, mu_e, mu_p):
    D, S, tau, Db, Sb, taub = q[0], q[1:4], q[4], q[5], q[6:9], q[9]
    B, E, psi, phi = q[10:13], q[13:16], q[16], q[17]
    ExB = _cross(E, B)
    St = [S[i] - ExB[i] for i in range(3)]
    taut = tau - (_dot(E, E) + _dot(B, B)) / 2
    mu = [mu_e, mu_p]
    # species split (Sec. 2.1.3)
    Ds = [(Db - mu_p * D) / (mu_e - mu_p), (Db - mu_e * D) / (mu_p - mu_e)]
    Ss = [[(Sb[i] - mu_p * St[i]) / (mu_e - mu_p) for i in range(3)],
          [(Sb[i] - mu_e * St[i]) / (mu_p - mu_e) for i in range(3)]]
    ts = [(taub - mu_p * taut) / (mu_e - mu_p), (taub - mu_e * taut) / (mu_p - mu_e)]
    sp = [_hydro_prims(Ds[k], Ss[k], ts[k], gamma) for k in range(2)]
    varrho = sum(mu[k] * sp[k][0] * sp[k][3] for k in range(2))
    J = [sum(mu[k] * sp[k][0] * sp[k][3] * sp[k][1][i] for k in range(2)) for i in range(3)]
    wp2 = sum(mu[k] ** 2 * sp[k][0] for k in range(2))
    Wb = sum(mu[k] ** 2 * sp[k][0] * sp[k][3] for k in range(2)) / wp2
    u = [sum(mu[k] ** 2 * sp[k][0] * sp[k][3] * sp[k][1][i] for k in range(2)) / wp2 for i in range(3)]
    varrho0 = Wb * varrho - _dot(J, u)
    eta = 1 / sigma
    uxB = _cross(u, B)
    s = [mp.mpf(0)] * 18
    for i in range(3):
        s[6 + i] = wp2 * (Wb * E[i] + uxB[i] - eta * (J[i] - varrho * u[i]))
        s[13 + i] = -J[i]
    s[9] = wp2 * (_dot(u, E) - eta * (varrho - varrho0 * Wb))
    s[16] = varrho - kappa * psi
    s[17] = -kappa * phi
    return s


def _full_solve(r, adt, source):
    """mpmath multidimensional Newton on G(q) = q - r - adt Psi(q), all N_c unknowns, from q = r."""
    n = len(r)
    rr = [mp.mpf(float(x)) for x in r]
    a = mp.mpf(adt)

    def Gfun(*q):
        s = source(list(q))
        return [q[i] - rr[i] - a * s[i] for i in range(n)]

    sol = mp.findroot(Gfun, rr, tol=mp.mpf(10) ** -30, maxsteps=60)
    return np.array([float(sol[i]) for i in range(n)])


@pytest.mark.parametrize("k,sigma", [(0, 10.0), (1, 1e3), (2, 1e5), (3, 1e3)])
def test_sf_stage_matches_full_system(k, sigma):
    mp.dps = 40
    s = WL.random_sf_states(4, seed=31, wmax=3.0)[k]
    gamma, adt = 4.0 / 3.0, G * 4e-3
    r = O.sf_p2c(s, 0.3, 0.05, -0.02, gamma)
    q, _ = O.sf_implicit(r, adt, gamma, sigma)
    ref = _full_solve(r, adt, lambda qq: _sf_source_full(qq, mp.mpf(gamma), mp.mpf(sigma), 1))
    scale = np.maximum(np.abs(ref), 1.0)
    assert np.max(np.abs(q - ref) / scale) <= 1e-12


@pytest.mark.parametrize("k,sigma", [(0, 1e4), (1, 1e2)])
def test_tf_stage_matches_full_system(k, sigma):
    mp.dps = 40
    s = WL.random_tf_states(2, seed=32, wmax=1.5, drift=0.01)[k]
    gamma, adt, mu_e, mu_p = 4.0 / 3.0, G * 5e-4, -1e3, 1e3
    r = O.tf_p2c(s, gamma, mu_e, mu_p, 0.02, -0.01)
    q, _ = O.tf_implicit(r, adt, gamma, sigma, mu_e, mu_p)
    ref = _full_solve(r, adt, lambda qq: _tf_source_full(qq, mp.mpf(gamma), mp.mpf(sigma), 1,
                                                         mp.mpf(mu_e), mp.mpf(mu_p)))
    scale = np.maximum(np.abs(ref), 1.0)
    assert np.max(np.abs(q - ref) / scale) <= 1e-12


def test_c2p_root_unique_and_matches():
    """The pressure residual has one sign change on (0, 2(tau~ + D) + 1] (scan
    on a log grid) and the oracle's root agrees with mpmath's bracketing solve."""
    mp.dps = 30
    for s in WL.random_sf_states(6, seed=33, wmax=5.0, theta=(1e-2, 1e2), emax=0.5, bmax=0.5):
        gamma = 5.0 / 3.0
        q = O.sf_p2c(s, 0.0, 0.0, 0.0, gamma)
        B, E = q[5:8], q[8:11]
        St = q[1:4] - np.cross(E, B)
        taut = q[4] - 0.5 * (E @ E + B @ B)
        D = q[0]
        S2 = mp.mpf(float(St @ St))

        def f(p):
            Z = taut + D + p
            W = 1 / mp.sqrt(1 - S2 / Z ** 2)
            rho = D / W
            eps = Z / (rho * W ** 2) - 1 - p / rho
            return (gamma - 1) * rho * eps - p

        grid = [mp.mpf(10) ** (mp.mpf(e) / 20) for e in range(-200, 60)]
        vals = [f(p) for p in grid if p < 2 * (taut + D) + 1]
        changes = sum(1 for a, b in zip(vals, vals[1:]) if (a > 0) != (b > 0))
        assert changes == 1
        rho, v, p, W = _hydro_prims(mp.mpf(float(D)), [mp.mpf(float(x)) for x in St], mp.mpf(float(taut)),
                                    mp.mpf(gamma))
        w = O.sf_c2p(q, gamma)
        assert abs(w[4] - float(p)) <= 1e-13 * float(p) + 1e-15
