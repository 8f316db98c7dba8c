"""Pins of the oracle's SSP3(332) IMEX step (Sec. 2.2.1, Table 2; no GPU):
the tableau's linear amplification on the uniform EM-decay problem (closed
form), its L-stability, and conservation on a periodic grid.

Table 2 with g = 1 - 1/sqrt(2): explicit rows (0,0,0), (1,0,0), (1/4,1/4,0);
implicit rows (g,0,0), (1-2g,g,0), (1/2-g,0,g); weights (1/6,1/6,2/3)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_09721_gb300 import workloads as WL

G = 1.0 - 1.0 / math.sqrt(2.0)


def ssp3_linear_decay_factor(z):
    """Amplification of y' = -k y over one SSP3(332) step, z = k dt (L = 0):
    y1 = y/(1+g z); y2 = (y - (1-2g) z y1)/(1+g z); y3 = (y - (1/2-g) z y1)/(1+g z);
    y^{n+1} = y - z (y1/6 + y2/6 + 2 y3/3)."""
    y1 = 1.0 / (1.0 + G * z)
    y2 = (1.0 - (1.0 - 2.0 * G) * z * y1) / (1.0 + G * z)
    y3 = (1.0 - (0.5 - G) * z * y1) / (1.0 + G * z)
    return 1.0 - z * (y1 / 6.0 + y2 / 6.0 + 2.0 * y3 / 3.0)


def test_ssp3_l_stable():
    """z -> inf: z y1 -> 1/g, z y2 -> (3g-1)/g^2, z y3 -> (2g-1/2)/g^2, so
    R(inf) = (6g^2 - 12g + 3)/(6g^2), which vanishes because g solves
    2g^2 - 4g + 1 = 0; R(z) also matches exp(-z) to second order."""
    assert abs(2 * G * G - 4 * G + 1) < 1e-15
    assert abs(ssp3_linear_decay_factor(1e12)) < 1e-10
    for z in (1e-2, 5e-3):
        assert abs(ssp3_linear_decay_factor(z) - math.exp(-z)) <= 0.2 * z ** 3


@pytest.mark.parametrize("sigma", [1e-3, 1.0, 1e2, 1e4, 1e8])
def test_ssp3_em_decay_closed_form(sigma):
    """Uniform state at rest, B = 0, varrho = 0, E != 0: L = 0 and J = sigma E,
    so E^{n+1} = R(sigma dt) E^n; psi, phi decay with R(kappa dt); tau is
    conserved, hence p = (Gamma - 1)(tau - E^2/2) exactly."""
    gamma, dt = 4.0 / 3.0, 0.01
    E0 = np.array([0.3, -0.2, 0.5])
    prim = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, *E0]
    sim = O.Sim(O.MODEL_SF, 6, 1, (0, 1), (0, 1), gamma, sigma, O.BC_PERIODIC, O.BC_PERIODIC, scheme=1)
    q0 = O.sf_p2c(prim, 0.0, 0.7, -0.4, gamma)
    sim.set_cons(np.ascontiguousarray(np.broadcast_to(q0[:, None, None], (14, 1, 6))))
    sim.step(dt, 1)
    q = sim.cons()
    RE, Rk = ssp3_linear_decay_factor(sigma * dt), ssp3_linear_decay_factor(dt)
    for i in range(3):
        assert np.max(np.abs(q[8 + i] - RE * E0[i])) <= 1e-13 * np.max(np.abs(E0))
    assert np.max(np.abs(q[12] - Rk * 0.7)) <= 1e-14
    assert np.max(np.abs(q[13] - Rk * -0.4)) <= 1e-14
    assert np.max(np.abs(q[4] - q0[4])) <= 1e-14
    p_exact = (gamma - 1.0) * (q0[4] - 0.5 * float(np.dot(RE * E0, RE * E0)))
    assert np.max(np.abs(sim.prims()[4] - p_exact)) <= 1e-13


def test_ssp3_conservation_periodic():
    wl = WL.khi(n=16, seed=5, sigma=1e3)
    sim = O.Sim(O.MODEL_SF, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y, scheme=1)
    sim.set_prims(wl.prims)
    c0 = sim.cons()
    a0 = np.abs(c0).reshape(14, -1).sum(axis=1)
    s0 = c0.reshape(14, -1).sum(axis=1)
    sim.step(wl.dt, 3)
    s1 = sim.cons().reshape(14, -1).sum(axis=1)
    for v in (0, 1, 2, 3, 4, 5, 6, 7, 11):
        assert abs(s1[v] - s0[v]) <= 1e-13 * max(a0[v], 1e-3 * wl.cells), (v, s1[v] - s0[v])


def test_ssp3_differs_from_ssp2_at_third_order_in_time():
    """On smooth KHI data the two integrators agree to O(dt^3) per step: the
    difference of one step shrinks ~8x when dt halves (a dropped or mis-weighted
    stage would leave an O(dt^2) or O(dt) difference)."""
    wl = WL.khi(n=16, seed=5, sigma=1.0, a=0.2)
    d = []
    for dt in (wl.dt, wl.dt / 2):
        out = []
        for scheme in (0, 1):
            sim = O.Sim(O.MODEL_SF, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
                        scheme=scheme)
            sim.set_prims(wl.prims)
            sim.step(dt, 1)
            out.append(sim.cons())
        d.append(np.abs(out[1] - out[0]).max())
    assert 5.0 <= d[0] / d[1] <= 12.0, d
