"""Pins of the differentiable oracle (oracle/autodiff_sf.py, PyTorch CPU, FP64)
that serves as the reference of the discrete adjoint: its forward run agrees
with the independent C oracle to round-off, and its autograd gradient agrees
with Richardson-extrapolated central differences of the C oracle's forward
map (accurate to ~1e-7: solver round-off over the step, and WENO3 weights
that vary on the sqrt(eps) ~ 1e-3 scale of the data's differences)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from conftest import parity_errors
from paper_1808_09721_gb300 import workloads as WL

A = pytest.importorskip("oracle.autodiff_sf")

CASES = [
    ("brio_wu_10", lambda: WL.brio_wu(nx=10), 3),
    ("field_loop_6x6", lambda: WL.field_loop(n=6, nsteps=3), 3),
    ("khi_6x6_stiff", lambda: WL.khi(n=6, seed=3, sigma=1e5), 3),
]


def c_oracle(wl, prims, nsteps, sigma=None):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma if sigma is None else sigma,
              wl.bc_x, wl.bc_y)
    o.set_prims(np.ascontiguousarray(prims))
    o.step(wl.dt, nsteps)
    return o.cons()


def ad(wl, lam, nsteps):
    return A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, lam)


@pytest.mark.parametrize("name,make,nsteps", CASES)
def test_forward_matches_c_oracle(name, make, nsteps):
    wl = make()
    lam = np.zeros((14,) + wl.prims.shape[1:])
    _, _, _, q = ad(wl, lam, nsteps)
    err = parity_errors(0, q, c_oracle(wl, wl.prims, nsteps))
    assert np.all(err <= 1e-12), (name, err)


def test_gradient_matches_c_oracle_differences():
    wl = WL.brio_wu(nx=10)
    nsteps = 3
    lam = np.random.default_rng(5).normal(size=(14,) + wl.prims.shape[1:])
    _, g, gs, _ = ad(wl, lam, nsteps)

    def J(prims, sigma=None):
        return float((lam * c_oracle(wl, prims, nsteps, sigma)).sum())

    fd = np.zeros_like(g)
    for v in range(11):
        h = 1e-5 * max(np.abs(wl.prims[v]).max(), 1e-2)
        for idx in np.ndindex(wl.prims.shape[1:]):
            def Jd(d):
                p = wl.prims.copy()
                p[(v,) + idx] += d
                return J(p)
            d1 = (Jd(h) - Jd(-h)) / (2 * h)
            d2 = (Jd(h / 2) - Jd(-h / 2)) / h
            fd[(v,) + idx] = (4 * d2 - d1) / 3
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()
    h = 1e-4 * wl.sigma
    d1 = (J(wl.prims, wl.sigma + h) - J(wl.prims, wl.sigma - h)) / (2 * h)
    d2 = (J(wl.prims, wl.sigma + h / 2) - J(wl.prims, wl.sigma - h / 2)) / h
    fs = (4 * d2 - d1) / 3
    assert abs(gs - fs) <= 1e-6 * abs(fs), (gs, fs)


def test_jvp_matches_c_oracle_differences():
    """The forward-mode derivative (reverse mode applied twice) along a random
    direction of the primitives and sigma, against Richardson-extrapolated
    central differences of the C oracle's final state."""
    wl = WL.field_loop(n=6, nsteps=3)
    nsteps = 3
    rng = np.random.default_rng(7)
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[:, None, None]
    vs = 0.1 * wl.sigma
    Jv = A.jvp(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, vp, vs)

    def q(h):
        return c_oracle(wl, wl.prims + h * vp, nsteps, wl.sigma + h * vs)
    # h = 1e-6: the field loop's near-constant fields make the WENO3 weights
    # vary fast (1e-5 leaves a 3e-6 truncation error); 1e-7 reaches round-off
    h = 1e-6
    d1 = (q(h) - q(-h)) / (2 * h)
    d2 = (q(h / 2) - q(-h / 2)) / h
    fd = (4 * d2 - d1) / 3
    assert np.abs(Jv - fd).max() <= 1e-7 * np.abs(fd).max(), np.abs(Jv - fd).max() / np.abs(fd).max()


def test_ssp3_forward_and_gradient_match_c_oracle():
    """SSP3(332) (Table 2): the differentiable oracle's forward run agrees with
    the C oracle's SSP3 step to round-off, and its gradient with central
    differences of the C oracle (Brio-Wu, 10 cells, 3 steps)."""
    wl = WL.brio_wu(nx=10)
    nsteps = 3

    def c3(prims, sigma=None):
        o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma if sigma is None else sigma,
                  wl.bc_x, wl.bc_y, scheme=1)
        o.set_prims(np.ascontiguousarray(prims))
        o.step(wl.dt, nsteps)
        return o.cons()
    lam = np.random.default_rng(6).normal(size=(14,) + wl.prims.shape[1:])
    _, g, gs, q = A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, lam,
                             scheme=1)
    assert np.all(parity_errors(0, q, c3(wl.prims)) <= 1e-12)
    rng = np.random.default_rng(8)
    for _ in range(3):
        d = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[:, None, None]
        h = 1e-6
        J = lambda t: float((lam * c3(wl.prims + t * d)).sum())
        d1 = (J(h) - J(-h)) / (2 * h)
        d2 = (J(h / 2) - J(-h / 2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(float((g * d).sum()) - fd) <= 1e-6 * abs(fd), (float((g * d).sum()), fd)
    h = 1e-4 * wl.sigma
    Js = lambda sg: float((lam * c3(wl.prims, sg)).sum())
    d1 = (Js(wl.sigma + h) - Js(wl.sigma - h)) / (2 * h)
    d2 = (Js(wl.sigma + h / 2) - Js(wl.sigma - h / 2)) / h
    fs = (4 * d2 - d1) / 3
    assert abs(gs - fs) <= 1e-6 * abs(fs), (gs, fs)


def test_3d_forward_and_gradient_match_c_oracle():
    """3-D grids: the differentiable oracle's step (z ghosts, Gauss's law and the
    flux divergence along z) agrees with the C oracle's 3-D step, and its
    gradient with directional central differences of it (random smooth fields
    on a 6 x 5 x 4 periodic grid, 2 steps)."""
    wl = WL.random_smooth((4, 5, 6), seed=5, sigma=30.0)
    nsteps = 2

    def c3d(prims, sigma=None):
        o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma if sigma is None else sigma,
                  wl.bc_x, wl.bc_y, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
        o.set_prims(np.ascontiguousarray(prims))
        o.step(wl.dt, nsteps)
        return o.cons()
    lam = np.random.default_rng(4).normal(size=(14,) + wl.prims.shape[1:])
    _, g, gs, q = A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, lam,
                             bcz=wl.bc_z, dz=wl.dz)
    assert np.all(parity_errors(0, q.reshape(14, -1, 1), c3d(wl.prims).reshape(14, -1, 1)) <= 1e-12)
    rng = np.random.default_rng(9)
    scale = np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[:, None, None, None]
    for _ in range(2):
        d = rng.normal(size=wl.prims.shape) * scale
        h = 1e-6
        J = lambda t: float((lam * c3d(wl.prims + t * d)).sum())
        d1 = (J(h) - J(-h)) / (2 * h)
        d2 = (J(h / 2) - J(-h / 2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(float((g * d).sum()) - fd) <= 1e-6 * abs(fd), (float((g * d).sum()), fd)
    h = 1e-4 * wl.sigma
    Js = lambda sg: float((lam * c3d(wl.prims, sg)).sum())
    fs = (4 * ((Js(wl.sigma + h / 2) - Js(wl.sigma - h / 2)) / h) - (Js(wl.sigma + h) - Js(wl.sigma - h)) / (2 * h)) / 3
    assert abs(gs - fs) <= 1e-6 * abs(fs), (gs, fs)
