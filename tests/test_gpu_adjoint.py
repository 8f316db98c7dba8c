"""Discrete adjoint of the SSP2(222) step (single fluid, FP64) through the C
ABI and the torch.autograd.Function: gradients of the final-state functional
J = sum (B_x^2 + B_y^2 + 2 B_z^2) dV (= integral of B_z^2 + |B|^2) with respect
to the initial primitives and sigma, checked against central finite
differences of the GPU forward run and of the CPU oracle."""
import dataclasses

import numpy as np
import pytest

import oracle as O
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


def functional_np(q, wl):
    dv = wl.dx * (wl.dy if wl.ny > 1 else 1.0)
    return float((q[5] ** 2 + q[6] ** 2 + 2.0 * q[7] ** 2).sum() * dv)


def gpu_J(Sim, wl, prims, nsteps):
    s = Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y, wl.cfl)
    s.set_prims(np.ascontiguousarray(prims))
    s.step(wl.dt, nsteps)
    s.check()
    return functional_np(s.cons(), wl)


def oracle_J(wl, prims, nsteps):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    o.set_prims(np.ascontiguousarray(prims))
    o.step(wl.dt, nsteps)
    return functional_np(o.cons(), wl)


def gradients(env, wl, nsteps, ckpt):
    torch, Sim, ImexSteps = env
    p0 = torch.tensor(wl.prims, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(wl.sigma, dtype=torch.float64, requires_grad=True)
    q = ImexSteps.apply(p0, sig, wl, nsteps, ckpt)
    dv = wl.dx * (wl.dy if wl.ny > 1 else 1.0)
    J = ((q[5] ** 2 + q[6] ** 2 + 2.0 * q[7] ** 2).sum() * dv)
    J.backward()
    return J.item(), p0.grad.cpu().numpy(), sig.grad.item()


def direction(wl, seed):
    """Smooth random perturbation of every primitive field, scaled to the field."""
    rng = np.random.default_rng(seed)
    d = np.zeros_like(wl.prims)
    ny, nx = wl.ny, wl.nx
    y, x = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    for v in range(11):
        a, b, c = rng.normal(size=3)
        shape = np.sin(2 * np.pi * (x + a)) * np.cos(2 * np.pi * (y + b)) + 0.3 * c
        scale = max(np.abs(wl.prims[v]).max(), 1e-3)
        d[v] = scale * shape
    return d


CASES = [
    ("field_loop", lambda: WL.field_loop(n=24, nsteps=12), 12, 5),
    ("brio_wu_1d", lambda: WL.brio_wu(nx=40), 10, 4),
    ("khi_stiff", lambda: WL.khi(n=16, seed=3, sigma=1e5), 6, 3),
]


@pytest.mark.parametrize("name,make,nsteps,ckpt", CASES)
def test_adjoint_matches_finite_differences(env, name, make, nsteps, ckpt):
    torch, Sim, _ = env
    wl = make()
    J, gp, gs = gradients(env, wl, nsteps, ckpt)
    assert abs(J - gpu_J(Sim, wl, wl.prims, nsteps)) <= 1e-14 * abs(J)
    # sigma: J is insensitive to sigma in the stiff limit (dJ/dsigma ~ 1/sigma^2),
    # so the difference step is 1e-3 sigma (truncation ~1e-6 relative) and the
    # bound includes the forward run's round-off floor (1e-13 |J|) divided by h
    h = 1e-3 * wl.sigma
    fd = (gpu_J(Sim, dataclasses.replace(wl, sigma=wl.sigma + h), wl.prims, nsteps) -
          gpu_J(Sim, dataclasses.replace(wl, sigma=wl.sigma - h), wl.prims, nsteps)) / (2 * h)
    assert abs(gs - fd) <= 1e-4 * abs(fd) + 1e-13 * abs(J) / h, (gs, fd)
    # initial primitives, two random directions
    for seed in (1, 2):
        d = direction(wl, seed)
        h = 1e-6
        fd = (gpu_J(Sim, wl, wl.prims + h * d, nsteps) - gpu_J(Sim, wl, wl.prims - h * d, nsteps)) / (2 * h)
        ad = float((gp * d).sum())
        assert abs(ad - fd) <= 1e-5 * abs(fd), (name, seed, ad, fd)


def test_adjoint_twenty_random_directions(env):
    """Central differences (h = 1e-6) of the GPU forward run along 20 random
    smooth directions of the initial primitives, each combined with a random
    relative change of sigma, against the adjoint's directional derivative
    (relative error <= 1e-5)."""
    torch, Sim, _ = env
    wl = WL.field_loop(n=24, nsteps=12)
    nsteps = 12
    J, gp, gs = gradients(env, wl, nsteps, 5)
    rng = np.random.default_rng(21)
    worst = 0.0
    for seed in range(100, 120):
        d = direction(wl, seed)
        ds = float(rng.uniform(-1.0, 1.0)) * 1e-2 * wl.sigma  # sigma direction (scaled like the fields)
        h = 1e-6
        jp = gpu_J(Sim, dataclasses.replace(wl, sigma=wl.sigma + h * ds), wl.prims + h * d, nsteps)
        jm = gpu_J(Sim, dataclasses.replace(wl, sigma=wl.sigma - h * ds), wl.prims - h * d, nsteps)
        fd = (jp - jm) / (2 * h)
        ad = float((gp * d).sum()) + gs * ds
        rel = abs(ad - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= 1e-5, (seed, ad, fd)
    print(f"20 directions: worst relative difference {worst:.2e}")


def test_adjoint_matches_oracle_finite_differences(env):
    """Directional derivatives of the oracle's FP64 run (central differences)
    agree with the GPU adjoint gradient."""
    wl = WL.field_loop(n=16, nsteps=8)
    nsteps = 8
    J, gp, gs = gradients(env, wl, nsteps, 3)
    assert abs(J - oracle_J(wl, wl.prims, nsteps)) <= 1e-9 * abs(J)
    for seed in (3, 4):
        d = direction(wl, seed)
        h = 1e-5
        fd = (oracle_J(wl, wl.prims + h * d, nsteps) - oracle_J(wl, wl.prims - h * d, nsteps)) / (2 * h)
        ad = float((gp * d).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd), (seed, ad, fd)
    h = 1e-3 * wl.sigma
    fd = (oracle_J(dataclasses.replace(wl, sigma=wl.sigma + h), wl.prims, nsteps) -
          oracle_J(dataclasses.replace(wl, sigma=wl.sigma - h), wl.prims, nsteps)) / (2 * h)
    assert abs(gs - fd) <= 1e-4 * abs(fd) + 1e-13 * abs(J) / h, (gs, fd)


def test_adjoint_restores_state_and_repeats(env):
    """The adjoint leaves the final state in place and can be called again."""
    torch, Sim, _ = env
    wl = WL.field_loop(n=12, nsteps=6)
    s = Sim.from_workload(wl)
    s.record(6, 4)
    s.step(wl.dt, 6)
    before = s.cons()
    lam = np.zeros_like(before)
    lam[5:8] = 2.0 * before[5:8] * np.array([1.0, 1.0, 2.0])[:, None, None]  # dJ/dB
    g1, s1 = s.adjoint(lam)
    np.testing.assert_array_equal(s.cons(), before)
    g2, s2 = s.adjoint(lam)
    # the face transposes accumulate with FP64 atomics: sums agree to round-off
    # of the largest entry, not bit for bit
    np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-12 * np.abs(g1).max())
    assert abs(s2 - s1) <= 1e-10 * abs(s1)


def test_failed_rearm_leaves_context_unarmed(env):
    """Arming again drops the earlier recording first; when the new arming
    fails (here: a caller workspace that is too small, refused on the host
    before any device work) the context is left unarmed: steps run without
    recording, bit for bit as an unrecorded run, and the adjoint is refused."""
    import ctypes as C
    from paper_1808_09721_gb300 import _lib as L
    torch, Sim, _ = env
    wl = WL.field_loop(n=12, nsteps=4)
    s = Sim.from_workload(wl)
    s.record(4, 2)
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    code = s.lib.rmhd_record(s.h, 4, 2, C.c_void_p(small.data_ptr()), 256)
    assert L.ERRORS.get(code) == "RMHD_ERR_NOMEM", code
    ref = Sim.from_workload(wl)
    s.step(wl.dt, 4)
    ref.step(wl.dt, 4)
    s.check()
    np.testing.assert_array_equal(s.cons(), ref.cons())
    with pytest.raises(L.RmhdError):
        s.adjoint(np.zeros((14,) + s.shape))


def oracle_lin_J(wl, prims, lam, nsteps):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    o.set_prims(np.ascontiguousarray(prims))
    o.step(wl.dt, nsteps)
    return float((lam * o.cons()).sum())


def oracle_gradient(wl, lam, nsteps, rel=1e-5):
    """Every entry of dJ/d(prims) of the oracle's forward run, J = sum lam * q,
    by Richardson-extrapolated central differences (steps rel and rel/2 of the
    field's magnitude). Accurate to ~1e-7 of max|g|: the solvers' round-off
    divided by the step, and the WENO3 weights vary on the sqrt(eps) ~ 1e-3
    scale of the data's differences, which bounds the step from above."""
    p = wl.prims
    g = np.zeros_like(p)
    for v in range(p.shape[0]):
        h = rel * max(np.abs(p[v]).max(), 1e-2)
        for idx in np.ndindex(p.shape[1:]):
            def J(d):
                q = p.copy()
                q[(v,) + idx] += d
                return oracle_lin_J(wl, q, lam, nsteps)
            d1 = (J(h) - J(-h)) / (2 * h)
            d2 = (J(h / 2) - J(-h / 2)) / h
            g[(v,) + idx] = (4 * d2 - d1) / 3
    return g


TINY = [
    ("brio_wu_10", lambda: WL.brio_wu(nx=10), 3, 2),
    ("field_loop_6x6", lambda: WL.field_loop(n=6, nsteps=3), 3, 2),
    ("khi_6x6_stiff", lambda: WL.khi(n=6, seed=3, sigma=1e5), 3, 2),
]


@pytest.mark.parametrize("name,make,nsteps,ckpt", TINY)
def test_adjoint_gradient_entrywise_vs_oracle(env, name, make, nsteps, ckpt):
    """Brute force on tiny grids: every entry of the GPU adjoint's gradient
    against the oracle's full difference gradient (the oracle's forward map,
    not the GPU's), for a random linear functional of the final state."""
    torch, Sim, _ = env
    wl = make()
    lam = np.random.default_rng(5).normal(size=(14,) + wl.prims.shape[1:])
    s = Sim.from_workload(wl)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, _ = s.adjoint(np.ascontiguousarray(lam))
    go = oracle_gradient(wl, lam, nsteps)
    err = np.abs(gp - go).max() / np.abs(go).max()
    assert err <= 2e-6, (name, err)


@pytest.mark.parametrize("name,make,nsteps,ckpt", TINY)
def test_adjoint_matches_autodiff_oracle(env, name, make, nsteps, ckpt):
    """The GPU adjoint against the exact gradient of the same discrete step
    from the differentiable oracle (reverse-mode autograd of a PyTorch-CPU FP64
    restatement, pinned to the C oracle): every entry of dJ/d(prims) and dJ/dsigma."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = make()
    lam = np.random.default_rng(5).normal(size=(14,) + wl.prims.shape[1:])
    s = Sim.from_workload(wl)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(lam))
    _, go, gso, _ = A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y,
                               wl.dx, wl.dy, lam)
    err = np.abs(gp - go).max() / np.abs(go).max()
    print(name, "entrywise relative error", err, "dJ/dsigma", gs, gso)
    assert err <= 1e-9, (name, err)
    assert abs(gs - gso) <= 1e-9 * abs(gso) + 1e-12 * np.abs(go).max(), (name, gs, gso)


@pytest.mark.parametrize("name,make,nsteps,ckpt", TINY)
def test_adjoint_dot_product(env, name, make, nsteps, ckpt):
    """<J v, w> = <v, J^T w>: the GPU adjoint (reverse mode, J^T w for a random
    w) against the differentiable oracle's forward-mode derivative J v (its
    reverse mode applied twice) along a random direction v of the initial
    primitives and sigma."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = make()
    rng = np.random.default_rng(17)
    w = rng.normal(size=(14,) + wl.prims.shape[1:])
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[
        (slice(None),) + (None,) * (wl.prims.ndim - 1)]
    vs = 0.1 * wl.sigma
    s = Sim.from_workload(wl)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(w))
    Jv = A.jvp(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, vp, vs)
    lhs = float((Jv * w).sum())
    rhs = float((gp * vp).sum() + gs * vs)
    # round-off of an inner product is relative to the magnitude of its terms
    mag = max(float(np.abs(Jv * w).sum()), float(np.abs(gp * vp).sum() + abs(gs * vs)))
    rel = abs(lhs - rhs) / mag
    print(name, "dot-product relative difference", rel)
    assert rel <= 1e-12, (name, lhs, rhs, rel)


@pytest.mark.parametrize("name,make,nsteps,ckpt", TINY)
def test_adjoint_ssp3_matches_autodiff_oracle(env, name, make, nsteps, ckpt):
    """SSP3(332) (Table 2; three implicit stages reversed from the third): every
    entry of the GPU gradient and dJ/dsigma against the differentiable oracle's
    SSP3 gradient (pinned to the C oracle's SSP3 step)."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = make()
    lam = np.random.default_rng(15).normal(size=(14,) + wl.prims.shape[1:])
    s = Sim.from_workload(wl, scheme=1)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(lam))
    _, go, gso, _ = A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y,
                               wl.dx, wl.dy, lam, scheme=1)
    err = np.abs(gp - go).max() / np.abs(go).max()
    print(name, "SSP3 entrywise relative error", err, "dJ/dsigma", gs, gso)
    assert err <= 1e-9, (name, err)
    assert abs(gs - gso) <= 1e-9 * abs(gso) + 1e-12 * np.abs(go).max(), (name, gs, gso)


@pytest.mark.parametrize("name,make,nsteps,ckpt", TINY)
def test_adjoint_ssp3_dot_product(env, name, make, nsteps, ckpt):
    """<J v, w> = <v, J^T w> for SSP3(332): GPU reverse mode against the
    differentiable oracle's forward-mode derivative."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = make()
    rng = np.random.default_rng(27)
    w = rng.normal(size=(14,) + wl.prims.shape[1:])
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[
        (slice(None),) + (None,) * (wl.prims.ndim - 1)]
    vs = 0.1 * wl.sigma
    s = Sim.from_workload(wl, scheme=1)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(w))
    Jv = A.jvp(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, vp, vs, scheme=1)
    lhs = float((Jv * w).sum())
    rhs = float((gp * vp).sum() + gs * vs)
    # round-off of an inner product is relative to the magnitude of its terms
    mag = max(float(np.abs(Jv * w).sum()), float(np.abs(gp * vp).sum() + abs(gs * vs)))
    rel = abs(lhs - rhs) / mag
    print(name, "SSP3 dot-product relative difference", rel)
    assert rel <= 1e-12, (name, lhs, rhs, rel)


def test_adjoint_ssp3_finite_differences(env):
    """SSP3(332) through the torch.autograd.Function: directional central
    differences of the GPU forward (field loop 24^2, 12 steps, checkpoints
    every 5) along random directions of the primitives and sigma."""
    torch, Sim, ImexSteps = env
    wl = WL.field_loop(n=24, nsteps=12)
    nsteps = 12
    p0 = torch.tensor(wl.prims, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(wl.sigma, dtype=torch.float64, requires_grad=True)
    q = ImexSteps.apply(p0, sig, wl, nsteps, 5, 1)
    dv = wl.dx * wl.dy
    J = (q[5] ** 2 + q[6] ** 2 + 2.0 * q[7] ** 2).sum() * dv
    J.backward()
    gp, gs = p0.grad.cpu().numpy(), sig.grad.item()

    def gJ(prims, sigma):
        s = Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, sigma, wl.bc_x, wl.bc_y, wl.cfl, scheme=1)
        s.set_prims(np.ascontiguousarray(prims))
        s.step(wl.dt, nsteps)
        s.check()
        return functional_np(s.cons(), wl)
    assert abs(J.item() - gJ(wl.prims, wl.sigma)) <= 1e-14 * abs(J.item())
    rng = np.random.default_rng(33)
    for seed in (41, 42, 43):
        d = direction(wl, seed)
        ds = float(rng.uniform(-1.0, 1.0)) * 1e-2 * wl.sigma
        h = 1e-6
        fd = (gJ(wl.prims + h * d, wl.sigma + h * ds) - gJ(wl.prims - h * d, wl.sigma - h * ds)) / (2 * h)
        ad = float((gp * d).sum()) + gs * ds
        assert abs(ad - fd) <= 1e-5 * abs(fd), (seed, ad, fd)


TINY3D = [
    ("random_3d", lambda: WL.random_smooth((4, 5, 6), seed=5, sigma=30.0), 2, 1, 0),
    ("khi3d", lambda: WL.khi3d(shape=(4, 5, 6), seed=3), 2, 1, 0),
    ("random_3d_ssp3", lambda: WL.random_smooth((4, 5, 6), seed=6, sigma=30.0), 2, 1, 1),
]


@pytest.mark.parametrize("name,make,nsteps,ckpt,scheme", TINY3D, ids=[c[0] for c in TINY3D])
def test_adjoint_3d_matches_autodiff_oracle(env, name, make, nsteps, ckpt, scheme):
    """3-D grids (z fluxes transposed face by face, Gauss's law along z in the
    initial map): every entry of the GPU gradient and dJ/dsigma against the
    differentiable oracle's 3-D gradient (pinned to the C oracle's 3-D step)."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = make()
    lam = np.random.default_rng(25).normal(size=(14,) + wl.prims.shape[1:])
    s = Sim.from_workload(wl, scheme=scheme)
    s.record(nsteps, ckpt)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(lam))
    _, go, gso, _ = A.gradient(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, lam,
                               scheme=scheme, bcz=wl.bc_z, dz=wl.dz)
    err = np.abs(gp - go).max() / np.abs(go).max()
    print(name, "3-D entrywise relative error", err, "dJ/dsigma", gs, gso)
    assert err <= 1e-9, (name, err)
    assert abs(gs - gso) <= 1e-9 * abs(gso) + 1e-12 * np.abs(go).max(), (name, gs, gso)


def test_adjoint_3d_dot_product(env):
    """<J v, w> = <v, J^T w> on a 3-D grid."""
    A = pytest.importorskip("oracle.autodiff_sf")
    torch, Sim, _ = env
    wl = WL.random_smooth((4, 5, 6), seed=7, sigma=30.0)
    nsteps = 2
    rng = np.random.default_rng(37)
    w = rng.normal(size=(14,) + wl.prims.shape[1:])
    vp = rng.normal(size=wl.prims.shape) * np.abs(wl.prims).reshape(11, -1).max(axis=1).clip(1e-2)[
        (slice(None),) + (None,) * (wl.prims.ndim - 1)]
    vs = 0.1 * wl.sigma
    s = Sim.from_workload(wl)
    s.record(nsteps, 1)
    s.step(wl.dt, nsteps)
    s.check()
    gp, gs = s.adjoint(np.ascontiguousarray(w))
    Jv = A.jvp(wl.prims, wl.sigma, wl.dt, nsteps, wl.gamma, wl.bc_x, wl.bc_y, wl.dx, wl.dy, vp, vs,
               bcz=wl.bc_z, dz=wl.dz)
    lhs = float((Jv * w).sum())
    rhs = float((gp * vp).sum() + gs * vs)
    # round-off of an inner product is relative to the magnitude of its terms
    mag = max(float(np.abs(Jv * w).sum()), float(np.abs(gp * vp).sum() + abs(gs * vs)))
    rel = abs(lhs - rhs) / mag
    print("3-D dot-product relative difference", rel)
    assert rel <= 1e-12, (lhs, rhs, rel)
