"""Discrete adjoint of the two-fluid IMEX step (FP64, SSP2(222) and SSP3(332))
through the C ABI: every entry of dJ/d(prims) (16 primitives per cell) and
dJ/dsigma of a random linear functional of the final state against the exact
gradient of the same discrete step from the two-fluid differentiable oracle
(oracle/autodiff_tf.py, pinned to the C oracle), the dot-product identity
<J v, w> = <v, J^T w> against the oracle's forward-mode derivative, and
directional differences of the GPU forward run.

Per stage the adjoint solves the transposed 7 x 7 system of the stiff
unknowns (Sbar, taubar, E) and differentiates the species split and the two
per-species pressure roots by the implicit-function theorem."""
import dataclasses

import numpy as np
import pytest

from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    _lib.load()
    from paper_1808_09721_gb300.adjoint import ImexSteps
    from paper_1808_09721_gb300.sim import Sim
    return torch, Sim, ImexSteps


TINY = [
    ("tf_brio_wu_10", lambda: WL.tf_brio_wu(nx=10), 3, 2, 0),
    ("tf_sheet_8x8", lambda: WL.tf_sheet(n=8, seed=1), 3, 2, 0),
    ("random_tf_6x8", lambda: WL.random_smooth((6, 8), seed=1, model=1, sigma=10.0, mu=20.0), 3, 2, 0),
    ("tf_brio_wu_10_ssp3", lambda: WL.tf_brio_wu(nx=10), 2, 1, 1),
    ("random_tf_5x6_ssp3", lambda: WL.random_smooth((5, 6), seed=3, model=1, sigma=30.0, mu=20.0), 2, 1, 1),
]
IDS = [c[0] for c in TINY]


def adjoint(Sim, wl, lam, nsteps, ckpt, scheme):
    s = Sim.from_workload(wl, scheme=scheme)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    return s, s.adjoint(np.ascontiguousarray(lam))


@pytest.mark.parametrize("name,make,nsteps,ckpt,scheme", TINY, ids=IDS)
def test_adjoint_matches_autodiff_oracle(env, name, make, nsteps, ckpt, scheme):
    A = pytest.importorskip("oracle.autodiff_tf")
    torch, Sim, _ = env
    wl = make()
    lam = np.random.default_rng(5).normal(size=(18,) + wl.prims.shape[1:])
    s, (gp, gs) = adjoint(Sim, wl, lam, nsteps, ckpt, scheme)
    assert gp.shape == wl.prims.shape
    _, go, gso, _ = A.gradient(wl, nsteps, lam, scheme=scheme)
    err = np.abs(gp - go).max() / np.abs(go).max()
    print(name, "entrywise relative error", err, "dJ/dsigma", gs, gso)
    assert err <= 1e-9, (name, err)
    assert abs(gs - gso) <= 1e-9 * abs(gso) + 1e-12 * np.abs(go).max(), (name, gs, gso)


# The dot-product identity compares the GPU's linearisation at its forward
# run with the oracle's at its own; their roots agree to round-off times the
# conditioning of the stage solves. For the stiff, under-resolved sheet above
# (mu = -+1e3, sigma = 1e4, a tanh sheet of width 0.05 on 8 cells) the two
# gradients agree entry by entry to ~1e-10 of max |g|, so a contraction with
# random vectors differs by ~1e-12 whatever the adjoint does (measured 4.5e-13
# to 9e-12 as the forward's rounding changes). The identity is checked at
# 1e-12 on a conditioned sheet (width 0.25, mu = -+1e2; the stiff one stays
# in the entrywise test).
DOT = [c if c[0] != "tf_sheet_8x8" else
       ("tf_sheet_8x8_resolved", lambda: WL.tf_sheet(n=8, seed=1, mu=1e2, width=0.25), 3, 2, 0) for c in TINY]


@pytest.mark.parametrize("name,make,nsteps,ckpt,scheme", DOT, ids=[c[0] for c in DOT])
def test_adjoint_dot_product(env, name, make, nsteps, ckpt, scheme):
    """<J v, w> = <v, J^T w>: GPU reverse mode against the oracle's forward-mode
    derivative along a random direction of the primitives and sigma."""
    A = pytest.importorskip("oracle.autodiff_tf")
    torch, Sim, _ = env
    wl = make()
    rng = np.random.default_rng(17)
    w = rng.normal(size=(18,) + wl.prims.shape[1:])
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(16, -1).max(axis=1).clip(1e-2)[
        (slice(None),) + (None,) * (wl.prims.ndim - 1)]
    vs = 0.1 * wl.sigma
    _, (gp, gs) = adjoint(Sim, wl, w, nsteps, ckpt, scheme)
    Jv = A.jvp(wl, nsteps, vp, vs, scheme=scheme)
    lhs = float((Jv * w).sum())
    rhs = float((gp * vp).sum() + gs * vs)
    # round-off of an inner product is relative to the magnitude of its terms
    mag = max(float(np.abs(Jv * w).sum()), float(np.abs(gp * vp).sum() + abs(gs * vs)))
    rel = abs(lhs - rhs) / mag
    print(name, "dot-product relative difference", rel)
    assert rel <= 1e-12, (name, lhs, rhs, rel)


def gpu_lin_J(Sim, wl, prims, lam, nsteps, sigma=None):
    s = Sim.from_workload(dataclasses.replace(wl, sigma=wl.sigma if sigma is None else sigma))
    s.set_prims(np.ascontiguousarray(prims))
    s.step(wl.dt, nsteps)
    s.check()
    return float((lam * s.cons()).sum())


def test_adjoint_directional_differences_of_gpu_forward(env):
    """Sheet 16^2, 6 steps, checkpoints every 4: the adjoint's directional
    derivative along smooth directions of the primitives and sigma against
    central differences (step 1e-6) of the GPU forward run. The directions
    move both species alike, so the plasma stays neutral to first order: a
    direction that separates charge changes Dbar by ~mu h and needs h ~ 1e-8
    before the WENO3 weights are linear over the step, where the stage
    solves' convergence floor divided by h dominates the difference (such
    directions are covered entry by entry against the oracle above)."""
    torch, Sim, _ = env
    wl = WL.tf_sheet(n=16, seed=2)
    nsteps = 6
    rng = np.random.default_rng(3)
    lam = rng.normal(size=(18, wl.ny, wl.nx))
    _, (gp, gs) = adjoint(Sim, wl, lam, nsteps, 4, 0)
    y, x = np.meshgrid(np.arange(wl.ny) / wl.ny, np.arange(wl.nx) / wl.nx, indexing="ij")
    for seed in (1, 2, 3):
        r = np.random.default_rng(seed)
        fields = [max(np.abs(wl.prims[v]).max(), 1e-3) * (np.sin(2 * np.pi * (x + r.normal()))
                  * np.cos(2 * np.pi * (y + r.normal())) + 0.3 * r.normal()) for v in range(16)]
        fields[5:10] = fields[0:5]  # positive species moves as the electrons
        d = np.stack(fields)
        ds = float(r.uniform(-1.0, 1.0)) * 1e-2 * wl.sigma
        h = 1e-6
        jp = gpu_lin_J(Sim, wl, wl.prims + h * d, lam, nsteps, wl.sigma + h * ds)
        jm = gpu_lin_J(Sim, wl, wl.prims - h * d, lam, nsteps, wl.sigma - h * ds)
        fd = (jp - jm) / (2 * h)
        ad = float((gp * d).sum()) + gs * ds
        assert abs(ad - fd) <= 1e-5 * abs(fd), (seed, ad, fd)


def test_adjoint_restores_state_and_repeats(env):
    torch, Sim, _ = env
    wl = WL.tf_sheet(n=12, seed=4)
    s = Sim.from_workload(wl)
    s.record(5, 3)
    s.step(wl.dt, 5)
    before = s.cons()
    lam = np.random.default_rng(8).normal(size=before.shape)
    g1, s1 = s.adjoint(lam)
    np.testing.assert_array_equal(s.cons(), before)
    g2, s2 = s.adjoint(lam)
    # face transposes accumulate with FP64 atomics: equal to round-off, not bit for bit
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-12 * np.abs(g1).max())
    assert abs(s2 - s1) <= 1e-10 * abs(s1)


def test_adjoint_autograd_function(env):
    """ImexSteps (torch.autograd.Function) returns the 16-plane gradient for a
    two-fluid workload and agrees with the C-ABI adjoint."""
    torch, Sim, ImexSteps = env
    wl = WL.tf_sheet(n=8, seed=5)
    nsteps = 3
    lam = np.random.default_rng(9).normal(size=(18, wl.ny, wl.nx))
    p0 = torch.tensor(wl.prims, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(wl.sigma, dtype=torch.float64, requires_grad=True)
    q = ImexSteps.apply(p0, sig, wl, nsteps, 2)
    (torch.tensor(lam, device="cuda") * q).sum().backward()
    _, (gp, gs) = adjoint(Sim, wl, lam, nsteps, 2, 0)
    np.testing.assert_allclose(p0.grad.cpu().numpy(), gp, rtol=0, atol=1e-12 * np.abs(gp).max())
    assert abs(sig.grad.item() - gs) <= 1e-10 * abs(gs)
