"""GPU diagnostics reduction (rmhd_diagnostics and rmhd_diagnostics_noalloc)
against sums of the FP64 CPU oracle's own state.

The diagnostics are the invariants of Sec. 2.1 (cell sums of D, tau, S_x, B_x
and the charge variable -- varrho for one fluid, Dbar for two fluids -- times
the cell volume), max |v| and the count of non-finite conserved values. Here
they are formed with NumPy from the oracle's conserved state and primitives
after the same steps, so a wrong variable index, a wrong species offset or a
missing volume factor (the grids have dx, dy, dz != 1) fails. The GPU and
oracle states differ at round-off (parity bar 1e-9 of each variable's natural
scale, measured ~1e-13), so each sum is compared within 1e-11 x (number of
cells) x (natural scale of the variable) x (cell volume).
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from conftest import parity_scale
from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

KEYS = ("sum_D", "sum_tau", "sum_Sx", "sum_Bx", "sum_charge", "max_v", "nonfinite")


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    lib = _lib.load()
    from paper_1808_09721_gb300.sim import Sim
    return torch, lib, Sim


def _oracle(wl):
    kw = {}
    if wl.nz > 1:
        kw = dict(nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    s = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, **kw)
    s.set_prims(wl.prims)
    return s


def _vol(wl, batch=False):
    if batch:
        return 1.0  # a batch sums over its runs' cells without a volume factor
    return wl.dx * (wl.dy if wl.ny > 1 else 1.0) * (wl.dz if wl.nz > 1 else 1.0)


def _oracle_diag(model, q, p, vol):
    """The seven diagnostics of a state from the oracle: q [N_c][...], p [n_prim][...]."""
    iB, iR = (5, 11) if model == 0 else (10, 5)
    sums = [q[v].sum() * vol for v in (0, 4, 1, iB, iR)]
    if model == 0:
        vmax = np.sqrt((p[1:4] ** 2).sum(axis=0)).max()
    else:
        vmax = max(np.sqrt((p[1:4] ** 2).sum(axis=0)).max(), np.sqrt((p[6:9] ** 2).sum(axis=0)).max())
    bad = float((~np.isfinite(q)).sum())
    return np.array(sums + [vmax, bad])


def _tolerances(model, q, vol, mu_ref):
    s = parity_scale(model, q.reshape(q.shape[0], -1, 1), mu_ref)
    iB, iR = (5, 11) if model == 0 else (10, 5)
    n = q[0].size
    return np.array([1e-11 * n * s[v] * vol for v in (0, 4, 1, iB, iR)])


def _check(model, got, want, tol):
    assert np.all(np.abs(got[:5] - want[:5]) <= tol), (got, want, tol)
    assert abs(got[5] - want[5]) <= 1e-12 * max(want[5], 1e-300), (got[5], want[5])
    assert got[6] == want[6] == 0.0


def _noalloc(torch, lib, sim, wl):
    cons = torch.empty((sim.nc,) + sim.shape, dtype=torch.float64, device=sim.device)
    prims = torch.empty((sim.np,) + sim.shape, dtype=torch.float64, device=sim.device)
    sim.cons(out=cons)
    sim.prims(out=prims)
    torch.cuda.synchronize(sim.device)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device=sim.device)
    st = torch.cuda.current_stream(sim.device)
    rc = lib.rmhd_diagnostics_noalloc(wl.model, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz,
                                      C.c_void_p(cons.data_ptr()), C.c_void_p(prims.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(st.cuda_stream))
    assert rc == 0
    st.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["khi_70x45", "tf_sheet_48", "khi3d_12", "brio_wu_400"])
def test_diagnostics_against_oracle_state(env, name):
    torch, lib, Sim = env
    wl = {"khi_70x45": lambda: WL.khi(n=70, ny=45, seed=4),
          "tf_sheet_48": lambda: WL.tf_sheet(n=48, seed=5),
          "khi3d_12": lambda: WL.khi3d(n=12, seed=6),
          "brio_wu_400": lambda: WL.brio_wu(nx=400)}[name]()
    mu_ref = max(abs(wl.mu_e), abs(wl.mu_p)) if wl.model == 1 else 1.0
    g = Sim.from_workload(wl)
    o = _oracle(wl)
    for steps in (0, 3):
        if steps:
            g.step(wl.dt, steps)
            g.check()
            o.step(wl.dt, steps)
        q, p = o.cons(), o.prims()
        want = _oracle_diag(wl.model, q, p, _vol(wl))
        tol = _tolerances(wl.model, q, _vol(wl), mu_ref)
        d = g.diagnostics()
        _check(wl.model, np.array([d[k] for k in KEYS]), want, tol)
        _check(wl.model, _noalloc(torch, lib, g, wl), want, tol)
        # the CFL step of the grid's directions
        h = min([wl.dx] + ([wl.dy] if wl.ny > 1 else []) + ([wl.dz] if wl.nz > 1 else []))
        assert abs(d["dt_cfl"] - wl.cfl * h) <= 1e-15 * h


def test_batch_diagnostics_against_oracle_runs(env):
    """A batch sums over all its runs' cells (no volume factor): the sum of the
    per-run sums of independent oracle runs."""
    torch, lib, Sim = env
    runs = WL.batch_tubes(count=7, seed=11, nmin=20, nmax=90)
    b = Sim.batch(runs)
    b.step(0.0, 4)
    b.check()
    parts, tols = [], []
    for w in runs:
        o = _oracle(w)
        o.step(w.dt, 4)  # each run's own CFL step, as the batch takes with dt <= 0
        q, p = o.cons(), o.prims()
        parts.append(_oracle_diag(0, q, p, 1.0))
        tols.append(_tolerances(0, q, 1.0, 1.0))
    want = np.array([sum(x[k] for x in parts) for k in range(5)] + [max(x[5] for x in parts), 0.0])
    tol = np.sum(tols, axis=0)
    d = b.diagnostics()
    _check(0, np.array([d[k] for k in KEYS]), want, tol)
