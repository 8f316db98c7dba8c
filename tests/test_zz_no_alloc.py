"""GPU test of rmhd_diagnostics_noalloc, the diagnostics entry point for
callers that cannot allocate device memory (code running while a memory pool
or arena owns the device, or a framework that forbids allocation after
start-up): it keeps its partial sums in a static device array instead of a
workspace. Called several times in a row through the C ABI, on both models,
on 1-D, 2-D and 3-D grids and on a grid of about a million cells (hundreds of
partial sums for the final combine), and checked against rmhd_diagnostics of a
context holding the same state. Collected last so that a failure here cannot
hide other tests in a stop-at-first-failure run."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _vol(wl):
    return wl.dx * (wl.dy if wl.ny > 1 else 1.0) * (wl.dz if wl.nz > 1 else 1.0)


def _sum_scales(sim, wl):
    """Sum of |terms| of each diagnostic sum (cell volume included): the scale
    against which the summation-order rounding of a sum is judged."""
    q = sim.cons()
    iB, iR = (5, 11) if wl.model == 0 else (10, 5)
    return np.array([np.abs(q[v]).sum() * _vol(wl) for v in (0, 4, 1, iB, iR)])


def _noalloc_call(lib, wl, cons, prims, torch, device):
    out = torch.full((7,), float("nan"), dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    rc = lib.rmhd_diagnostics_noalloc(wl.model, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz,
                                      C.c_void_p(cons.data_ptr()), C.c_void_p(prims.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()
    return out.cpu().numpy()


def _noalloc(lib, sim, wl, torch):
    shape = sim.shape
    cons = torch.empty((sim.nc,) + shape, dtype=torch.float64, device=sim.device)
    prims = torch.empty((sim.np,) + shape, dtype=torch.float64, device=sim.device)
    sim.cons(out=cons)
    sim.prims(out=prims)
    torch.cuda.synchronize(sim.device)
    return _noalloc_call(lib, wl, cons, prims, torch, sim.device), cons, prims


def test_noalloc_diagnostics_match_context_diagnostics():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    lib = _lib.load()
    from paper_1808_09721_gb300.sim import Sim

    cases = [WL.khi(n=70, ny=45, seed=4), WL.tf_sheet(n=48, seed=5), WL.brio_wu(nx=400),
             WL.khi3d(n=12, seed=6), WL.khi(n=1024, seed=0)]
    for wl in cases:  # calls in a row: different models, dimensions and sizes
        sim = Sim.from_workload(wl)
        sim.step(wl.dt, 2)
        sim.check()
        ref = sim.diagnostics()
        want = np.array([ref[k] for k in ("sum_D", "sum_tau", "sum_Sx", "sum_Bx", "sum_charge", "max_v",
                                            "nonfinite")])
        scale = _sum_scales(sim, wl)
        for _ in range(2):  # the shared scratch keeps the last call's partials
            got, cons, prims = _noalloc(lib, sim, wl, torch)
            assert np.all(np.abs(got[:5] - want[:5]) <= 1e-12 * scale), (wl.name, got, want)
            assert got[5] == want[5] and got[6] == want[6] == 0.0, wl.name

    # non-finite values made on the host in a caller-owned array are counted
    wl = WL.khi(n=70, ny=45, seed=4)
    sim = Sim.from_workload(wl)
    _, cons, prims = _noalloc(lib, sim, wl, torch)
    host = cons.cpu().numpy()
    host[3, 5, 7] = np.nan
    host[9, 44, 69] = np.inf
    host[0, 0, 0] = -np.inf
    bad = torch.from_numpy(host).to(sim.device)
    got = _noalloc_call(lib, wl, bad, prims, torch, sim.device)
    assert got[6] == 3.0, got

    # beyond the static scratch (16,777,216 cells): rejected before any device work
    rc = lib.rmhd_diagnostics_noalloc(0, 8192, 4096, 1, 1e-3, 1e-3, 1.0, C.c_void_p(1), C.c_void_p(1),
                                      C.c_void_p(1), None)
    assert rc == -6
    # a 3-D grid needs ny > 1
    rc = lib.rmhd_diagnostics_noalloc(0, 8, 1, 4, 1e-3, 1e-3, 1e-3, C.c_void_p(1), C.c_void_p(1), C.c_void_p(1),
                                      None)
    assert rc == -1
