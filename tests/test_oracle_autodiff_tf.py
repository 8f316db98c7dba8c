"""Pins of the two-fluid differentiable oracle (oracle/autodiff_tf.py, PyTorch
CPU, FP64), the reference of the two-fluid discrete adjoint: its forward run
agrees with the independent C oracle to round-off (1-D, 2-D, SSP3), and its
autograd gradient agrees with Richardson-extrapolated central differences of
the C oracle's forward map.

Difference steps. With mu = 1e3 a change h of one species' density or pressure
moves the charge density Dbar by ~mu h; the WENO3 weights vary on the
sqrt(eps_WENO) ~ 1e-3 scale of the data's differences, so the step must keep
mu h well below that: h = 1e-7 of the field's magnitude (the truncation of a
1e-5 step reaches 10% in these variables). The solvers' round-off divided by h
then bounds the agreement at ~1e-7 of max |g|."""
import numpy as np
import pytest

import oracle as O
from conftest import parity_errors
from paper_1808_09721_gb300 import workloads as WL

A = pytest.importorskip("oracle.autodiff_tf")

FORWARD = [
    ("tf_brio_wu_12", lambda: WL.tf_brio_wu(nx=12), 3, 0),
    ("tf_sheet_8x8", lambda: WL.tf_sheet(n=8, seed=1), 3, 0),
    ("random_tf_6x8", lambda: WL.random_smooth((6, 8), seed=1, model=1, sigma=10.0, mu=20.0), 3, 0),
    ("tf_brio_wu_10_ssp3", lambda: WL.tf_brio_wu(nx=10), 2, 1),
]


def c_oracle(wl, prims, nsteps, sigma=None, scheme=0):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma if sigma is None else sigma,
              wl.bc_x, wl.bc_y, mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, scheme=scheme)
    o.set_prims(np.ascontiguousarray(prims))
    o.step(wl.dt, nsteps)
    return o.cons()


@pytest.mark.parametrize("name,make,nsteps,scheme", FORWARD, ids=[c[0] for c in FORWARD])
def test_forward_matches_c_oracle(name, make, nsteps, scheme):
    wl = make()
    q = A.forward(wl, nsteps, scheme)
    err = parity_errors(1, q, c_oracle(wl, wl.prims, nsteps, scheme=scheme))
    assert np.all(err <= 1e-12), (name, err)


def test_initial_map_matches_c_oracle():
    """Eq. (twoFluid cons) cell by cell against the C oracle's map."""
    import torch
    wl = WL.random_smooth((5, 7), seed=4, model=1, mu=50.0)
    q = A.prims_to_cons(torch.tensor(wl.prims), wl.gamma, (wl.mu_e, wl.mu_p)).numpy()
    for j, i in np.ndindex(wl.ny, wl.nx):
        ref = O.tf_p2c(wl.prims[:, j, i], wl.gamma, wl.mu_e, wl.mu_p)
        np.testing.assert_allclose(q[:, j, i], ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def _richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def test_gradient_matches_c_oracle_differences():
    """Every entry of dJ/d(prims) and dJ/dsigma of a random linear functional
    of the final state (two-fluid Brio-Wu tube, 10 cells, 2 steps)."""
    wl = WL.tf_brio_wu(nx=10)
    nsteps = 2
    lam = np.random.default_rng(5).normal(size=(18,) + wl.prims.shape[1:])
    _, g, gs, _ = A.gradient(wl, nsteps, lam)

    def J(prims, sigma=None):
        return float((lam * c_oracle(wl, prims, nsteps, sigma)).sum())

    fd = np.zeros_like(g)
    for v in range(16):
        h = 1e-7 * max(np.abs(wl.prims[v]).max(), 1e-2)
        for idx in np.ndindex(wl.prims.shape[1:]):
            def Jd(d):
                p = wl.prims.copy()
                p[(v,) + idx] += d
                return J(p)
            fd[(v,) + idx] = _richardson(Jd, h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()
    fs = _richardson(lambda d: J(wl.prims, wl.sigma + d), 1e-4 * wl.sigma)
    assert abs(gs - fs) <= 1e-6 * abs(fs), (gs, fs)


def test_gradient_2d_sampled_entries():
    """A 2-D grid (y fluxes, periodic wrap in both directions): 24 sampled
    entries of dJ/d(prims) against differences of the C oracle."""
    wl = WL.random_smooth((5, 6), seed=2, model=1, sigma=10.0, mu=20.0)
    nsteps = 2
    rng = np.random.default_rng(9)
    lam = rng.normal(size=(18,) + wl.prims.shape[1:])
    _, g, _, _ = A.gradient(wl, nsteps, lam)

    def J(prims):
        return float((lam * c_oracle(wl, prims, nsteps)).sum())

    for _ in range(24):
        idx = tuple(int(rng.integers(0, n)) for n in wl.prims.shape)
        h = 1e-6 * max(np.abs(wl.prims[idx[0]]).max(), 1e-2)

        def Jd(d):
            p = wl.prims.copy()
            p[idx] += d
            return J(p)
        assert abs(g[idx] - _richardson(Jd, h)) <= 1e-6 * np.abs(g).max(), idx


def test_jvp_matches_c_oracle_differences():
    """The forward-mode derivative (reverse mode applied twice) along a random
    direction of the primitives and sigma."""
    wl = WL.tf_brio_wu(nx=10)
    nsteps = 2
    rng = np.random.default_rng(7)
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(16, -1).max(axis=1).clip(1e-2)[:, None, None]
    vs = 0.1 * wl.sigma
    Jv = A.jvp(wl, nsteps, vp, vs)
    # every density moves at once along this direction: a smaller step than
    # for single entries keeps the charge separation within the WENO3 scale
    h = 1e-8
    fd = _richardson(lambda d: c_oracle(wl, wl.prims + d * vp, nsteps, wl.sigma + d * vs), h)
    assert np.abs(Jv - fd).max() <= 1e-6 * np.abs(fd).max()


def c_oracle_3d(wl, prims, nsteps):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y, mu_e=wl.mu_e,
              mu_p=wl.mu_p, kappa=wl.kappa, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    o.set_prims(np.ascontiguousarray(prims))
    o.step(wl.dt, nsteps)
    return o.cons()


def test_3d_forward_and_sampled_gradient():
    """A 3-D grid (z fluxes, ghosts along z): the forward run against the C
    oracle's 3-D step and 12 sampled gradient entries against its differences."""
    wl = WL.random_smooth((4, 5, 6), seed=2, model=1, sigma=10.0, mu=20.0)
    nsteps = 2
    rng = np.random.default_rng(11)
    lam = rng.normal(size=(18,) + wl.prims.shape[1:])
    _, g, _, q = A.gradient(wl, nsteps, lam)
    ref = c_oracle_3d(wl, wl.prims, nsteps)
    err = parity_errors(1, q.reshape(18, -1, 1), ref.reshape(18, -1, 1))
    assert np.all(err <= 1e-12), err

    def Jd(idx, d):
        p = wl.prims.copy()
        p[idx] += d
        return float((lam * c_oracle_3d(wl, p, nsteps)).sum())

    for _ in range(12):
        idx = tuple(int(rng.integers(0, n)) for n in wl.prims.shape)
        h = 1e-6 * max(np.abs(wl.prims[idx[0]]).max(), 1e-2)
        assert abs(g[idx] - _richardson(lambda d: Jd(idx, d), h)) <= 1e-6 * np.abs(g).max(), idx


@pytest.mark.parametrize("mistake", ["flux_sign", "split_swap", "source_eta"])
def test_planted_mistakes_fail_the_forward_pin(monkeypatch, mistake):
    """The forward pin catches plausible mistakes planted in the two-fluid
    autodiff oracle: a sign flip in the momentum flux's EM stress, the two
    species of the split swapped, eta = sigma instead of 1/sigma."""
    import torch
    wl = WL.random_smooth((5, 6), seed=3, model=1, sigma=10.0, mu=20.0)
    good = A.forward(wl, 1)
    if mistake == "flux_sign":
        orig = A.flux

        def flux(q, w, gamma, mu, j):
            f = orig(q, w, gamma, mu, j)
            E, B = q[A.E0:A.E0 + 3], q[A.B0:A.B0 + 3]
            return f.index_add(0, torch.arange(A.S0, A.S0 + 3), 2.0 * (E * E[j] + B * B[j]))
        monkeypatch.setattr(A, "flux", flux)
    elif mistake == "split_swap":
        orig = A.species_split
        monkeypatch.setattr(A, "species_split", lambda q, mu: tuple(reversed(orig(q, mu))))
    else:
        orig = A.source
        monkeypatch.setattr(A, "source", lambda q, w, sigma, kappa, mu: orig(q, w, 1.0 / sigma, kappa, mu))
    try:
        bad = A.forward(wl, 1)
    except ArithmeticError:
        return  # the planted mistake breaks the recovery or the stage solve outright
    err = parity_errors(1, bad, c_oracle(wl, wl.prims, 1))
    assert np.max(err) > 1e-6, (mistake, err)
    assert np.max(parity_errors(1, good, c_oracle(wl, wl.prims, 1))) <= 1e-12
