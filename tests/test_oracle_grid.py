"""Pins of the CPU oracle's grid step (no GPU): closed forms of the SSP2(222)
IMEX step, the ideal-MHD limit, conservation, rotational symmetry, and the
convergence of the WENO3/LF flux divergence.

Paper: Wright & Hawke, arXiv:1808.09721 -- Sec. 2.2.1 + Table 1 (SSP2(222)),
Sec. 2.1.1 (Ohm's law, divergence cleaning), Sec. 2.2.2 (flux splitting).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_09721_gb300 import workloads as WL

G = 1.0 - 1.0 / math.sqrt(2.0)


def ssp2_linear_decay_factor(z):
    """Amplification of y' = -k y over one SSP2(222) step, z = k dt, with the
    implicit tableau of Table 1: y1 = y/(1+g z); y2 = (y - (1-2g) z y1)/(1+g z);
    y^{n+1} = y - z/2 (y1 + y2)."""
    y1 = 1.0 / (1.0 + G * z)
    y2 = (1.0 - (1.0 - 2.0 * G) * z * y1) / (1.0 + G * z)
    return 1.0 - 0.5 * z * (y1 + y2)


def _uniform_cons(nx, ny, prim, varrho=0.0, psi=0.0, phi=0.0, gamma=4.0 / 3.0):
    q = O.sf_p2c(prim, varrho, psi, phi, gamma)
    return np.ascontiguousarray(np.broadcast_to(q[:, None, None], (14, ny, nx)))


def test_l_stable_limit_of_tableau():
    """4 g - 1 = 2 g^2 for g = 1 - 1/sqrt(2), hence R(inf) = 0 (L-stability)."""
    assert abs((4 * G - 1) - 2 * G * G) < 1e-15
    assert abs(ssp2_linear_decay_factor(1e12)) < 1e-10


@pytest.mark.parametrize("sigma", [1e-3, 1.0, 1e2, 1e4, 1e8])
def test_em_decay_closed_form(sigma):
    """Uniform state at rest with B = 0, varrho = 0, E != 0: L = 0 and J = sigma E
    (Ohm's law at v = 0), so E^{n+1} = R(sigma dt) E^n; psi and phi decay with
    R(kappa dt) (divergence cleaning, kappa = 1); tau is conserved so
    p = (Gamma - 1)(tau - E^2/2) exactly (Joule heating)."""
    gamma, dt = 4.0 / 3.0, 0.01
    E0 = np.array([0.3, -0.2, 0.5])
    prim = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, *E0]
    sim = O.Sim(O.MODEL_SF, 6, 1, (0, 1), (0, 1), gamma, sigma, O.BC_PERIODIC, O.BC_PERIODIC)
    cons = _uniform_cons(6, 1, prim, psi=0.7, phi=-0.4, gamma=gamma)
    sim.set_cons(cons)
    tau0 = cons[4, 0, 0]
    sim.step(dt, 1)
    q = sim.cons()
    RE, Rk = ssp2_linear_decay_factor(sigma * dt), ssp2_linear_decay_factor(1.0 * dt)
    E1 = RE * E0
    for i in range(3):
        assert np.max(np.abs(q[8 + i] - E1[i])) <= 1e-13 * np.max(np.abs(E0))
    assert np.max(np.abs(q[12] - Rk * 0.7)) <= 1e-14
    assert np.max(np.abs(q[13] - Rk * -0.4)) <= 1e-14
    assert np.max(np.abs(q[4] - tau0)) <= 1e-14
    assert np.max(np.abs(q[1:4])) == 0.0
    w = sim.prims()
    p_exact = (gamma - 1.0) * (tau0 - 0.5 * float(np.dot(E1, E1)))
    assert np.max(np.abs(w[4] - p_exact)) <= 1e-13
    assert np.max(np.abs(w[1:4])) == 0.0


def test_ideal_limit_slope():
    """Stiff limit of one implicit stage (Sec. 2.1.1: sigma -> inf is ideal RMHD):
    |E + v x B| after the solve falls like 1/(sigma a dt) -- slope -1 per decade."""
    prim = [1.0, 0.3, 0.2, -0.1, 1.0, 0.5, -0.7, 0.4, 0.0, 0.0, 0.0]
    r = O.sf_p2c(prim, 0.0, 0.0, 0.0, 5.0 / 3.0)
    adt = G * 1e-2
    res = []
    sigmas = [1e4, 1e5, 1e6, 1e7, 1e8]
    for sigma in sigmas:
        q, w = O.sf_implicit(r, adt, 5.0 / 3.0, sigma)
        v, B, E = w[1:4], q[5:8], q[8:11]
        res.append(np.linalg.norm(E + np.cross(v, B)))
    slopes = np.diff(np.log10(res)) / np.diff(np.log10(sigmas))
    assert np.all(np.abs(slopes + 1.0) < 0.05), slopes
    # and E.v -> 0 (no field along the flow in the ideal limit)
    assert abs(np.dot(w[1:4], q[8:11])) < 1e-6


def test_implicit_stage_fixed_point():
    """The stage solution satisfies q = r + a dt Psi(q) on every component (Eq. implicit
    stage): source-free components are r exactly, E, psi, phi to round-off."""
    states = WL.random_sf_states(40, seed=21, wmax=3.0)
    for k, s in enumerate(states):
        r = O.sf_p2c(s, 0.1 * (k % 3), 0.05, -0.02, 4.0 / 3.0)
        for sigma in (10.0, 1e4, 1e6):
            adt = G * 2e-3
            q, w = O.sf_implicit(r, adt, 4.0 / 3.0, sigma)
            src = O.sf_source(q, w, sigma)
            res = q - r - adt * src
            assert np.all(q[[0, 1, 2, 3, 4, 5, 6, 7, 11]] == r[[0, 1, 2, 3, 4, 5, 6, 7, 11]])
            scale = np.abs(q[8:11]).max() + adt * sigma * np.abs(q[8:11]).max() * 1e-3 + 1e-3
            assert np.max(np.abs(res[8:14])) <= 1e-13 * max(1.0, adt * sigma) * scale


def test_tf_implicit_stage_fixed_point():
    """Two-fluid stage (unknowns Sbar, taubar, E; Appendix A source) satisfies
    q = r + a dt Psi(q) with all other components equal to r."""
    states = WL.random_tf_states(20, seed=22, wmax=2.0, drift=0.01)
    for s in states:
        r = O.tf_p2c(s, 4.0 / 3.0, -1e3, 1e3, 0.03, -0.01)
        for sigma in (1e2, 1e4):
            adt = G * 1e-3
            q, w = O.tf_implicit(r, adt, 4.0 / 3.0, sigma, -1e3, 1e3)
            src = O.tf_source(q, w, sigma, -1e3, 1e3)
            res = q - r - adt * src
            assert np.all(q[[0, 1, 2, 3, 4, 5, 10, 11, 12]] == r[[0, 1, 2, 3, 4, 5, 10, 11, 12]])
            scale = np.abs(q).max()
            assert np.max(np.abs(res)) <= 1e-12 * scale


def _sums(q):
    return q.reshape(q.shape[0], -1).sum(axis=1)


def test_conservation_periodic_single_fluid():
    """On a periodic grid the flux differences telescope and D, S, tau, B, varrho
    have no source: their totals change only by round-off (Eq. resistive RMHD)."""
    wl = WL.khi(n=16, seed=5, sigma=1e3)
    sim = O.Sim(O.MODEL_SF, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    sim.set_prims(wl.prims)
    s0 = _sums(sim.cons())
    a0 = np.abs(sim.cons()).reshape(14, -1).sum(axis=1)
    sim.step(wl.dt, 3)
    s1 = _sums(sim.cons())
    for v in (0, 1, 2, 3, 4, 5, 6, 7, 11):
        assert abs(s1[v] - s0[v]) <= 1e-13 * max(a0[v], 1e-3 * wl.cells), (v, s1[v] - s0[v])


def test_conservation_periodic_two_fluid():
    """Two fluids: D, S, tau, Dbar and B totals are conserved on a periodic grid."""
    wl = WL.tf_sheet(n=12, seed=6, sigma=1e4)
    sim = O.Sim(O.MODEL_TF, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
                mu_e=wl.mu_e, mu_p=wl.mu_p)
    sim.set_prims(wl.prims)
    c0 = sim.cons()
    s0, a0 = _sums(c0), np.abs(c0).reshape(18, -1).sum(axis=1)
    sim.step(wl.dt, 2)
    s1 = _sums(sim.cons())
    for v in (0, 1, 2, 3, 4, 5, 10, 11, 12):
        assert abs(s1[v] - s0[v]) <= 1e-13 * max(a0[v], 1e-3 * wl.cells), (v, s1[v] - s0[v])


def _cyc(vec3):
    """Cyclic relabelling x->y, y->z, z->x of a 3-vector field (a proper rotation)."""
    return np.stack([vec3[2], vec3[0], vec3[1]])


def test_rotational_symmetry_x_vs_y():
    """A 1-D shock tube run along x equals the same tube run along y after the
    cyclic relabelling of vector components (the flux of Eq. resistive RMHD is
    covariant under rotations)."""
    wl = WL.brio_wu(nx=40)
    p = wl.prims[:, 0, :]  # (11, nx)
    ny_triv = 4
    px = np.repeat(p[:, None, :], ny_triv, axis=1)
    sx = O.Sim(O.MODEL_SF, 40, ny_triv, (0, 1), (0, 0.1), wl.gamma, wl.sigma, O.BC_OUTFLOW, O.BC_PERIODIC)
    sx.set_prims(px)
    py = np.concatenate([p[0:1], _cyc(p[1:4]), p[4:5], _cyc(p[5:8]), _cyc(p[8:11])])
    py = np.repeat(py[:, :, None], ny_triv, axis=2)
    sy = O.Sim(O.MODEL_SF, ny_triv, 40, (0, 0.1), (0, 1), wl.gamma, wl.sigma, O.BC_PERIODIC, O.BC_OUTFLOW)
    sy.set_prims(py)
    dt = 0.4 * (1.0 / 40) * 0.25  # both grids share dt = cfl * min(dx, dy)
    sx.step(dt, 5)
    sy.step(dt, 5)
    qx, qy = sx.cons()[:, 0, :], sy.cons()[:, :, 0]
    qx_rot = np.concatenate([qx[0:1], _cyc(qx[1:4]), qx[4:5], _cyc(qx[5:8]), _cyc(qx[8:11]), qx[11:14]])
    scale = np.maximum(np.abs(qx_rot).max(axis=1, keepdims=True), 1e-12)
    assert np.max(np.abs(qx_rot - qy) / scale) <= 1e-13


def test_flux_divergence_converges_on_smooth_data():
    """L = -d f/dx on smooth data: psi = exp(x) with E = 0 gives L[E_x] = -exp(x)
    (the E_x flux is psi, Eq. resistive RMHD). WENO3 with Jiang-Shu weights is
    second order at least on smooth monotone data; constant data gives L = 0."""
    errs = []
    ns = [32, 64, 128, 256]
    for n in ns:
        sim = O.Sim(O.MODEL_SF, n, 1, (0.0, 1.0), (0.0, 1.0), 4.0 / 3.0, 10.0, O.BC_OUTFLOW, O.BC_OUTFLOW)
        x = (np.arange(n) + 0.5) / n
        cons = _uniform_cons(n, 1, [1.0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0, 0]).copy()
        cons[12, 0, :] = np.exp(x)
        sim.set_cons(cons)
        L = sim.flux_divergence()
        interior = slice(3, n - 3)
        errs.append(np.max(np.abs(L[8, 0, interior] + np.exp(x[interior]))))
        # no other component sees psi except E_x (and nothing sees it at all in D, S, tau, B)
        assert np.max(np.abs(L[0:8])) == 0.0
    rates = np.diff(np.log(errs)) / -np.diff(np.log(ns))
    assert np.all(rates > 1.9), rates


def test_constant_state_has_zero_divergence():
    """Uniform state: every face flux is equal, so L = 0 exactly."""
    prim = [0.8, 0.3, -0.2, 0.1, 2.0, 0.3, 0.4, -0.5, 0.1, 0.2, -0.3]
    sim = O.Sim(O.MODEL_SF, 8, 8, (0, 1), (0, 1), 4.0 / 3.0, 1e3, O.BC_PERIODIC, O.BC_PERIODIC)
    sim.set_cons(_uniform_cons(8, 8, prim, 0.2, 0.1, 0.05))
    assert np.max(np.abs(sim.flux_divergence())) == 0.0


def test_periodic_wrap_narrower_than_stencil():
    """Periodic boundary condition: ghosts wrap modulo the extent, also when a
    direction has fewer cells than ghost layers. A 1-cell-wide periodic x
    direction is uniform along x, so the run equals the same data with 3
    identical copies along x."""
    wl = WL.khi(n=8, seed=2)
    p1 = np.ascontiguousarray(wl.prims[:, :, :1])
    p3 = np.ascontiguousarray(np.repeat(p1, 3, axis=2))
    out = []
    for p, nx in ((p1, 1), (p3, 3)):
        s = O.Sim(O.MODEL_SF, nx, 8, (0, nx / 8), (-0.5, 0.5), wl.gamma, wl.sigma, O.BC_PERIODIC, O.BC_PERIODIC)
        s.set_prims(p)
        s.step(wl.dt, 2)
        out.append(s.cons())
    assert np.all(np.isfinite(out[0]))
    np.testing.assert_array_equal(out[0][:, :, 0], out[1][:, :, 1])
