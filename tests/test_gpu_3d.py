"""3-D grids (nz > 1, one fluid) on the GPU through the C ABI against the
oracle's 3-D step: x-y flux pass per z-plane into a buffer, then the z pass on
x-z slabs with the stage combinations. Same bars as 2-D: relative L-infinity
<= 1e-9 (natural scale) FP64, relative L1 <= 1e-4 mixed."""
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


def oracle_for(wl, scheme=0):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              kappa=wl.kappa, scheme=scheme, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    o.set_prims(wl.prims)
    return o


def run_pair(Sim, wl, nsteps, precision=0, scheme=0):
    g = Sim.from_workload(wl, precision=precision, scheme=scheme)
    o = oracle_for(wl, scheme)
    g.step(wl.dt, nsteps)
    g.check()
    o.step(wl.dt, nsteps)
    return g, o


@pytest.mark.parametrize("shape,steps", [((16, 16, 16), 4), ((10, 12, 37), 3)])
def test_khi3d_parity(Sim, shape, steps):
    """Cubic grid and a ragged one (tiles of 32 x 8 do not fill x or y, and
    the x-z slabs do not fill z)."""
    wl = WL.khi3d(shape=shape, seed=1)
    g, o = run_pair(Sim, wl, steps)
    err = parity_errors(0, g.cons().reshape(14, -1, 1), o.cons().reshape(14, -1, 1))
    assert np.all(err <= TOL), err
    gp, op = g.prims(), o.prims()
    assert np.max(np.abs(gp - op)) <= 1e-9 * np.max(np.abs(op))


def test_khi3d_set_prims_gauss_law(Sim):
    """varrho = div E with the z term (second-order central differences)."""
    wl = WL.khi3d(shape=(6, 8, 10), seed=2)
    g = Sim.from_workload(wl)
    o = oracle_for(wl)
    np.testing.assert_allclose(g.cons()[11], o.cons()[11], rtol=0, atol=1e-13)


def test_tube_along_z_matches_oracle_and_x_tube(Sim):
    """A Brio-Wu tube along z (outflow in z, 4 x 4 periodic cross-section) against
    the oracle, and against the GPU's own tube along x after rotating the
    vector components (x -> z)."""
    n, m = 64, 4
    bw = WL.brio_wu(nx=n)
    p = bw.prims[:, 0, :]
    rot = lambda v: np.stack([v[1], v[2], v[0]])
    pz = np.concatenate([p[0:1], rot(p[1:4]), p[4:5], rot(p[5:8]), rot(p[8:11])])
    prims = np.ascontiguousarray(np.broadcast_to(pz[:, :, None, None], (11, n, m, m)))
    wl = WL.Workload("tube_z", 0, m, m, (0, 0.25), (0, 0.25), bw.gamma, bw.sigma, 1, 1, bw.cfl, 20, prims,
                     nz=n, zlim=(0.0, 1.0), bc_z=0)
    dt = bw.dt * 0.5
    g = Sim.from_workload(wl)
    o = oracle_for(wl)
    g.step(dt, 20)
    g.check()
    o.step(dt, 20)
    assert np.all(parity_errors(0, g.cons().reshape(14, -1, 1), o.cons().reshape(14, -1, 1)) <= TOL)
    gx = Sim.from_workload(bw)
    gx.step(dt, 20)
    qx = gx.cons()[:, 0, :]
    want = np.concatenate([qx[0:1], rot(qx[1:4]), qx[4:5], rot(qx[5:8]), rot(qx[8:11]), qx[11:14]])
    qz = g.cons()[:, :, 0, 0]
    scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-12)
    assert np.max(np.abs(qz - want) / scale) <= 1e-12


def test_khi3d_ssp3_and_mixed(Sim):
    wl = WL.khi3d(n=12, seed=3)
    g, o = run_pair(Sim, wl, 3, scheme=1)
    assert np.all(parity_errors(0, g.cons().reshape(14, -1, 1), o.cons().reshape(14, -1, 1)) <= TOL)
    g, o = run_pair(Sim, wl, 3, precision=1)
    want = o.cons()
    l1 = np.abs(g.cons() - want).reshape(14, -1).mean(axis=1) / parity_scale(0, want.reshape(14, -1, 1))
    assert np.all(l1 <= 1e-4), l1


@pytest.mark.parametrize("shape", [(2, 3, 5), (3, 2, 1), (5, 9, 2)])
def test_tiny_3d_grids(Sim, shape):
    """Degenerate 3-D grids: extents smaller than the stencil, a single cell
    across x, outflow along z."""
    wl = WL.khi3d(shape=shape, seed=4)
    import dataclasses
    wl = dataclasses.replace(wl, bc_z=0)
    g, o = run_pair(Sim, wl, 2)
    err = parity_errors(0, g.cons().reshape(14, -1, 1), o.cons().reshape(14, -1, 1))
    assert np.all(err <= TOL), err


def test_two_fluid_3d(Sim):
    """Two-fluid model on a 3-D grid (18 variables, z pass with the two-fluid
    flux along z): FP64 parity and the mixed form's L1 error."""
    wl = WL.tf_sheet3d(shape=(8, 12, 10), seed=3)
    g = Sim.from_workload(wl)
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    o.set_prims(wl.prims)
    g.step(wl.dt, 3)
    g.check()
    o.step(wl.dt, 3)
    want = o.cons()
    err = parity_errors(1, g.cons().reshape(18, -1, 1), want.reshape(18, -1, 1), 1e3)
    assert np.all(err <= TOL), err
    gm = Sim.from_workload(wl, precision=1)
    gm.step(wl.dt, 3)
    gm.check()
    l1 = np.abs(gm.cons() - want).reshape(18, -1).mean(axis=1) / parity_scale(1, want.reshape(18, -1, 1), 1e3)
    assert np.all(l1 <= 1e-4), l1
