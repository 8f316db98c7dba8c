"""Stage-solve robustness at very stiff conductivity and high Lorentz factor,
and the restart path of the solve, against the FP64 CPU oracle.

The implicit stage (Sec. 2.2.1, Eq. implicit stage) is a per-cell root whose
value does not depend on the start of the iteration. The GPU solve tries
three starts (the explicit part's E; the ideal-MHD limit E = -v x B,
Sec. 2.1.1; a continuation in a dt); the oracle restarts the same way.
Workloads: smooth random fields in bulk motion with Lorentz factor ~10 and
sigma up to 1e10 (a dt sigma W ~ 1e9), and Brio-Wu tubes at sigma 1e8 and
1e10.

Parity bar. D, S, tau, B: relative L-infinity 1e-9 of each variable's natural
scale. E, varrho, psi, phi: the same plus the round-off the method itself
amplifies at stiff sigma. Both implementations evaluate the current
J = varrho v + sigma W [E + v x B - (v.E) v] at the converged stage state,
where the bracket has cancelled to O(1/(a dt sigma W)) of its terms (|E|,
|v||B|, |v.E||v|, all O(1) here); its absolute round-off, a few units of
u = 2^-53 of those terms, is multiplied by sigma W and enters E through the
source term dt Psi_E = -dt J and varrho through the flux divergence of J
(dt/dx <= 1 here). Per step that is ~u sigma W dt of the field scale, which
no FP64 implementation can avoid: the bar for these variables is
1e-9 + 64 u sigma W_max dt n_steps (at sigma = 1e10, W = 11, dt = 5e-3,
3 steps: 3e-6; measured 3.8e-6 for varrho at K ~ 21).
`rmhd_set_first_start` makes every solve begin at start 1 or 2, so the
restart path is checked on whole grids, not only where start 0 happens to
fail; the solver statistics report which start converged."""
import numpy as np
import pytest

import oracle as O
from conftest import parity_errors
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


def _tolerance(wl, nsteps):
    """Per-variable bar (14 conserved variables): 1e-9, plus for E, varrho,
    psi, phi the amplified round-off of the stiff current (module docstring)."""
    v = wl.prims[1:4]
    wmax = float(np.max(1.0 / np.sqrt(1.0 - (v * v).sum(axis=0))))
    tol = np.full(14, TOL)
    tol[8:14] += 64 * 2.0 ** -53 * wl.sigma * wmax * wl.dt * nsteps
    return tol


def _oracle(wl, nsteps):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    o.set_prims(wl.prims)
    o.step(wl.dt, nsteps)
    return o.cons()


def _gpu(Sim, wl, nsteps, first=0):
    g = Sim.from_workload(wl)
    g.set_first_start(first)
    g.set_solver_stats(True)
    g.step(wl.dt, nsteps)
    g.check()
    st = g.solver_stats()
    return g.cons(), st


def _assert_all_solved(st, nsolves, first=0):
    starts = st["starts"]
    assert sum(starts.values()) == nsolves, starts
    assert starts["failed"] == 0, starts
    if first == 1:
        assert starts["explicit"] == 0 and starts["ideal_limit"] + starts["continuation"] == nsolves, starts
    if first == 2:
        assert starts["explicit"] == 0 and starts["ideal_limit"] == 0, starts


@pytest.mark.parametrize("sigma", [1e8, 1e10])
def test_relativistic_stiff_fields(Sim, sigma):
    wl = WL.relativistic_smooth((40, 32), seed=1, sigma=sigma, wmax=10.0, cfl=0.2)
    v = wl.prims[1:4]
    assert np.max(1.0 / np.sqrt(1.0 - (v * v).sum(axis=0))) > 10.0
    got, st = _gpu(Sim, wl, 3)
    err = parity_errors(0, got, _oracle(wl, 3))
    assert np.all(err <= _tolerance(wl, 3)), err
    assert np.all(err[:8] <= TOL), err  # D, S, tau, B at the plain bar
    _assert_all_solved(st, 2 * 3 * wl.cells)
    print(f"sigma={sigma:g}: starts {st['starts']}, rel err hydro/B {err[:8].max():.2e}, "
          f"E/charge {err[8:].max():.2e} (bar {_tolerance(wl, 3)[8]:.1e})")


@pytest.mark.parametrize("sigma", [1e8, 1e10])
def test_stiff_tubes(Sim, sigma):
    wl = WL.brio_wu(nx=200, sigma=sigma)
    got, st = _gpu(Sim, wl, 30)
    err = parity_errors(0, got, _oracle(wl, 30))
    assert np.all(err <= _tolerance(wl, 30)), err
    assert np.all(err[:8] <= TOL), err
    _assert_all_solved(st, 2 * 30 * wl.cells)


@pytest.mark.parametrize("first", [1, 2])
def test_restart_path_converges_to_the_same_root(Sim, first):
    for wl in (WL.khi(n=24, ny=20, seed=3), WL.relativistic_smooth((40, 32), seed=2, sigma=1e4, wmax=5.0),
               WL.brio_wu(nx=100, sigma=1e6)):
        got, st = _gpu(Sim, wl, 3, first)
        err = parity_errors(0, got, _oracle(wl, 3))
        assert np.all(err <= TOL), (wl.name, err)
        _assert_all_solved(st, 2 * 3 * wl.cells, first)


def test_first_start_control_is_validated(Sim):
    wl = WL.khi(n=16, seed=1)
    g = Sim.from_workload(wl)
    from paper_1808_09721_gb300._lib import RmhdError
    with pytest.raises(RmhdError):
        g.set_first_start(3)
    g.set_first_start(0)
    tf = Sim.from_workload(WL.tf_sheet(n=8, seed=1))
    with pytest.raises(RmhdError):
        tf.set_first_start(1)
