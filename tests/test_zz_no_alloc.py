"""GPU test of rmhd_diagnostics_noalloc, the diagnostics entry point for
callers that cannot allocate device memory (it keeps its partial sums in a
static device array instead of a workspace). Called twice in a row through the
C ABI, on different models and sizes, and checked against rmhd_diagnostics of
a context holding the same state. Collected last so that a failure here cannot
hide other tests in a stop-at-first-failure run."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _sum_scales(sim, wl):
    """Sum of |terms| of each diagnostic sum (cell volume included): the scale
    against which the summation-order rounding of a sum is judged."""
    q = sim.cons()
    vol = wl.dx * (wl.dy if wl.ny > 1 else 1.0)
    iB, iR = (5, 11) if wl.model == 0 else (10, 5)
    return np.array([np.abs(q[v]).sum() * vol for v in (0, 4, 1, iB, iR)])


def _noalloc(lib, sim, wl, torch):
    np_ = sim.np
    cons = torch.empty((sim.nc, wl.ny, wl.nx), dtype=torch.float64, device=sim.device)
    prims = torch.empty((np_, wl.ny, wl.nx), dtype=torch.float64, device=sim.device)
    sim.cons(out=cons)
    sim.prims(out=prims)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device=sim.device)
    stream = torch.cuda.current_stream(sim.device)
    rc = lib.rmhd_diagnostics_noalloc(wl.model, wl.nx, wl.ny, wl.dx, wl.dy, C.c_void_p(cons.data_ptr()),
                                      C.c_void_p(prims.data_ptr()), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_diagnostics_match_context_diagnostics():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    lib = _lib.load()
    from paper_1808_09721_gb300.sim import Sim

    cases = [WL.khi(n=70, ny=45, seed=4), WL.tf_sheet(n=48, seed=5)]
    for wl in cases:  # two calls in a row, different models and sizes
        sim = Sim.from_workload(wl)
        sim.step(wl.dt, 2)
        sim.check()
        ref = sim.diagnostics()
        got = _noalloc(lib, sim, wl, torch)
        want = np.array([ref[k] for k in ("sum_D", "sum_tau", "sum_Sx", "sum_Bx", "sum_charge", "max_v",
                                            "nonfinite")])
        scale = _sum_scales(sim, wl)
        assert np.all(np.abs(got[:5] - want[:5]) <= 1e-12 * scale), (got, want)
        assert got[5] == want[5] and got[6] == want[6] == 0.0

    # beyond the static scratch (16,777,216 cells): rejected before any device work
    rc = lib.rmhd_diagnostics_noalloc(0, 8192, 4096, 1e-3, 1e-3, C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), None)
    assert rc == -6
