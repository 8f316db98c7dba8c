"""SSP3(332) IMEX step (Sec. 2.2.1, Table 2) on the GPU through the C ABI
against the FP64 oracle's SSP3(332): the same bars as SSP2(222) -- relative
L-infinity <= 1e-9 (natural scale) in FP64, relative L1 <= 1e-4 mixed."""
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


def run_pair(Sim, wl, nsteps, precision=0):
    g = Sim.from_workload(wl, precision=precision, scheme=1)
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, scheme=1)
    o.set_prims(wl.prims)
    g.step(wl.dt, nsteps)
    g.check()
    o.step(wl.dt, nsteps)
    return g, o


def test_ssp3_brio_wu_full_run(Sim):
    wl = WL.brio_wu()
    g, o = run_pair(Sim, wl, wl.nsteps)
    err = parity_errors(0, g.cons(), o.cons())
    assert np.all(err <= TOL), err


@pytest.mark.parametrize("n,ny,steps", [(64, 64, 6), (70, 45, 4)])
def test_ssp3_khi(Sim, n, ny, steps):
    wl = WL.khi(n=n, ny=ny, seed=1)
    g, o = run_pair(Sim, wl, steps)
    assert np.all(parity_errors(0, g.cons(), o.cons()) <= TOL)
    gp, op = g.prims(), o.prims()
    assert np.max(np.abs(gp - op)) <= 1e-9 * np.max(np.abs(op))


def test_ssp3_two_fluid_sheet(Sim):
    wl = WL.tf_sheet(n=40, seed=2)
    g, o = run_pair(Sim, wl, 4)
    assert np.all(parity_errors(1, g.cons(), o.cons(), 1e3) <= TOL)


def test_ssp3_stiff_tubes(Sim):
    for wl in WL.batch_tubes(count=3, seed=5, nmin=100, nmax=300):
        g, o = run_pair(Sim, wl, 20)
        err = parity_errors(0, g.cons(), o.cons())
        assert np.all(err <= TOL), (wl.name, wl.sigma, err)


def test_ssp3_mixed_precision(Sim):
    wl = WL.khi(n=64, seed=1)
    g, o = run_pair(Sim, wl, 6, precision=1)
    want = o.cons()
    l1 = np.abs(g.cons() - want).reshape(14, -1).mean(axis=1) / parity_scale(0, want)
    assert np.all(l1 <= 1e-4), l1


def test_adjoint_refused_outside_its_scope(Sim):
    """The discrete adjoint covers the FP64 step of either model (both schemes):
    arming it on a mixed-precision SSP3(332) context, or on a grid with fewer
    than 3 cells along a direction, is an error, and the context stays usable."""
    from paper_1808_09721_gb300 import _lib as L
    for wl, prec in ((WL.field_loop(n=8, nsteps=2), 1), (WL.tf_sheet(n=8, seed=1, ny=2), 0)):
        s = Sim.from_workload(wl, scheme=1, precision=prec)
        with pytest.raises(L.RmhdError):
            s.record(2, 1)
        s.step(wl.dt, 1)
        s.check()
