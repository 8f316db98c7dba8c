"""Random smooth fields with every component nonzero (all three of v, B and E,
plus a resistive current), on the GPU through the C ABI against the oracle.

In the flux kernels the Maxwell components (B, E, psi, phi) are reconstructed
in pairs whose partner and sign depend on the direction (x, y, and z in the
3-D z pass); with every field component of order one, a wrong partner or sign
in any pair, direction or block would show at order one. Bars as elsewhere:
relative L-infinity <= 1e-9 of the natural scale (FP64), mean relative error
<= 1e-4 (mixed)."""
import numpy as np
import pytest

import oracle as O
from conftest import parity_errors, parity_scale
from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def Sim():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    _lib.load()
    from paper_1808_09721_gb300.sim import Sim as S
    return S


def run_pair(Sim, wl, nsteps, precision=0, scheme=0):
    g = Sim.from_workload(wl, precision=precision, scheme=scheme)
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, scheme=scheme, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    o.set_prims(wl.prims)
    g.step(wl.dt, nsteps)
    g.check()
    o.step(wl.dt, nsteps)
    nc = 14 if wl.model == 0 else 18
    return g.cons().reshape(nc, -1, 1), o.cons().reshape(nc, -1, 1)


CASES = [
    ("1d_periodic", (70,), 0, WL.PERIODIC),
    ("2d_periodic", (33, 45), 0, WL.PERIODIC),
    ("2d_outflow", (33, 45), 0, WL.OUTFLOW),
    ("3d_periodic", (10, 12, 18), 0, WL.PERIODIC),
    ("3d_outflow", (9, 10, 35), 0, WL.OUTFLOW),
    ("tf_2d_periodic", (24, 40), 1, WL.PERIODIC),
    ("tf_3d_periodic", (6, 10, 12), 1, WL.PERIODIC),
    # ragged 16 x 16 tiles of the line-sweep kernel in both directions, outflow
    ("tf_2d_outflow", (27, 35), 1, WL.OUTFLOW),
    ("tf_3d_outflow", (7, 19, 17), 1, WL.OUTFLOW),
]


@pytest.mark.parametrize("name,shape,model,bc", CASES, ids=[c[0] for c in CASES])
def test_random_fields_fp64(Sim, name, shape, model, bc):
    wl = WL.random_smooth(shape, seed=11, model=model, bc=bc)
    got, want = run_pair(Sim, wl, 3)
    err = parity_errors(model, got, want, 1e3 if model == 1 else 1.0)
    assert np.all(err <= TOL), (name, err)


@pytest.mark.parametrize("name,shape,model,bc", [CASES[1], CASES[3], CASES[5]], ids=["2d", "3d", "tf_2d"])
def test_random_fields_ssp3_fp64(Sim, name, shape, model, bc):
    wl = WL.random_smooth(shape, seed=12, model=model, bc=bc)
    got, want = run_pair(Sim, wl, 2, scheme=1)
    err = parity_errors(model, got, want, 1e3 if model == 1 else 1.0)
    assert np.all(err <= TOL), (name, err)


@pytest.mark.parametrize("name,shape,model,bc", [CASES[0], CASES[1], CASES[3], CASES[5]],
                         ids=["1d", "2d", "3d", "tf_2d"])
def test_random_fields_mixed(Sim, name, shape, model, bc):
    wl = WL.random_smooth(shape, seed=13, model=model, bc=bc)
    got, want = run_pair(Sim, wl, 3, precision=1)
    mu_ref = 1e3 if model == 1 else 1.0
    l1 = np.abs(got - want).reshape(got.shape[0], -1).mean(axis=1) / parity_scale(model, want, mu_ref)
    assert np.all(l1 <= 1e-4), (name, l1)


@pytest.mark.parametrize("name,shape,model,sigma", [
    ("1d_weakly_coupled", (70,), 0, 1e-2), ("2d_weakly_coupled", (33, 45), 0, 1e-2),
    ("1d_very_stiff", (70,), 0, 1e7), ("2d_very_stiff", (33, 45), 0, 1e7),
    ("3d_very_stiff", (8, 10, 12), 0, 1e7), ("tf_2d_very_stiff", (24, 40), 1, 1e7),
], ids=lambda x: x if isinstance(x, str) else None)
def test_random_fields_conductivity_limits(Sim, name, shape, model, sigma):
    """The weakly coupled (sigma dt << 1: Maxwell nearly decoupled from the
    fluid) and very stiff (sigma dt >> 1: near the ideal limit, where the
    explicit stages' J = sigma W (E + v x B - ...) multiplies any error of the
    stage's E by ~sigma dt) regimes of the implicit stage, with every field
    component of order one. (Two fluids at sigma <= 1 with these O(1) species
    currents are left out: there the oracle's stage solve finds no root either.)"""
    wl = WL.random_smooth(shape, seed=21, model=model, sigma=sigma)
    got, want = run_pair(Sim, wl, 3)
    err = parity_errors(model, got, want, 1e3 if model == 1 else 1.0)
    assert np.all(err <= TOL), (name, sigma, err)


@pytest.mark.parametrize("name,model,shape", [("sf_2d", 0, (12, 40)), ("sf_3d", 0, (6, 8, 40)),
                                              ("tf_2d", 1, (12, 40))])
def test_uniform_state_stays_uniform(Sim, name, model, shape):
    """Degenerate case: a uniform state (ideal E = -v x B, no current) on a
    periodic grid stays uniform -- every cell bit for bit equal to every other,
    the same arithmetic in every tile and at every tile edge -- and equal to
    the oracle's."""
    wl = WL.random_smooth(shape, seed=23, model=model)
    p = wl.prims.reshape(wl.prims.shape[0], -1)
    p[:] = p[:, [137]]  # the primitives of one cell everywhere
    nv = 14 if model == 0 else 18
    if model == 0:
        v, B = p[1:4, 0], p[5:8, 0]
        p[8:11] = -np.cross(v, B)[:, None]
    got, want = run_pair(Sim, wl, 4)
    assert np.all(got == got[:, :1, :]), name  # bitwise uniform
    err = parity_errors(model, got, want, 1e3 if model == 1 else 1.0)
    assert np.all(err <= TOL), (name, err)
    assert got.shape[0] == nv
