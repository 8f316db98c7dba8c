"""Domain decomposition along y on one GPU: slab contexts of one 2-D grid,
stepped phase by phase with the halo rows exchanged before every flux pass,
against the undecomposed run of the same grid. Each cell's update depends only
on the staged stencil values, so with correct halos the rows must agree bit
for bit (FP64, mixed and float-float flux forms, SSP2(222) and SSP3(332),
both models, periodic and outflow boundaries, uneven slabs). Also the
phase-by-phase stepping of an ordinary context against rmhd_imex_step, and
the refusals of the decomposition's calls.

The paper names multi-GPU runs as future work (Sec. 3.1, Sec. 5)."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    _lib.load()
    from paper_1808_09721_gb300 import slabs
    from paper_1808_09721_gb300.sim import Sim
    return Sim, slabs, _lib


def _pair(mods, wl, rows, nsteps, precision=0, scheme=0):
    Sim, slabs, _ = mods
    ref = Sim.from_workload(wl, precision=precision, scheme=scheme)
    state0 = ref.get_state()
    dec = slabs.LocalSlabs(wl, rows, precision=precision, scheme=scheme)
    dec.set_state(state0)
    ref.step(wl.dt, nsteps)
    ref.check()
    dec.step(wl.dt, nsteps)
    dec.check()
    return ref, dec


@pytest.mark.parametrize("case", ["khi_2", "khi_3_uneven", "khi_1_self"])
def test_slabs_match_undecomposed_periodic(mods, case):
    wl = WL.khi(n=64, seed=1)
    rows = {"khi_2": [32, 32], "khi_3_uneven": [20, 25, 19], "khi_1_self": [64]}[case]
    ref, dec = _pair(mods, wl, rows, 8)
    assert np.array_equal(dec.get_state(), ref.get_state())
    assert np.array_equal(dec.cons(), ref.cons())


def test_slabs_match_undecomposed_outflow(mods):
    """Outflow along y: the outer sides of the first and last slab are global
    boundaries (no halo); x periodic in one case, outflow in the other."""
    wl = WL.random_smooth((41, 36), seed=3, bc=WL.OUTFLOW, sigma=50.0)
    ref, dec = _pair(mods, wl, [13, 17, 11], 6)
    assert np.array_equal(dec.get_state(), ref.get_state())
    wl2 = wl.with_prims(wl.prims, bc_x=WL.PERIODIC)
    ref, dec = _pair(mods, wl2, [2, 37, 2], 6)
    assert np.array_equal(dec.get_state(), ref.get_state())


@pytest.mark.parametrize("precision,scheme", [(1, 0), (2, 0), (0, 1), (1, 1)])
def test_slabs_match_undecomposed_forms(mods, precision, scheme):
    wl = WL.khi(n=48, ny=40, seed=2)
    ref, dec = _pair(mods, wl, [16, 24], 5, precision, scheme)
    assert np.array_equal(dec.get_state(), ref.get_state())


@pytest.mark.parametrize("precision", [0, 1])
def test_slabs_two_fluids(mods, precision):
    wl = WL.tf_sheet(n=32, seed=3)
    ref, dec = _pair(mods, wl, [11, 21], 4, precision)
    assert np.array_equal(dec.get_state(), ref.get_state())
    # diagnostics of the slabs add up to the whole grid's
    d = [s.diagnostics() for s in dec.slabs]
    dr = ref.diagnostics()
    for k in ("sum_D", "sum_tau", "sum_Sx", "sum_Bx"):
        assert abs(sum(x[k] for x in d) - dr[k]) <= 1e-12 * max(abs(dr[k]), 1e-3), k


def test_dist_slab_single_rank_is_its_own_neighbour(mods):
    """DistSlab with one rank of a periodic grid: the exchange is a local copy
    of the slab's own rows (no process group needed)."""
    Sim, slabs, _ = mods
    wl = WL.khi(n=40, ny=24, seed=4)
    ref = Sim.from_workload(wl)
    st = ref.get_state()
    d = slabs.DistSlab(wl, 0, 1)
    d.slab.set_state(st)
    ref.step(wl.dt, 4)
    d.step(wl.dt, 4)
    d.slab.check()
    assert np.array_equal(d.slab.get_state(), ref.get_state())


def test_phase_stepping_equals_imex_step(mods):
    """rmhd_step_phase on an ordinary context: the phases of a step give
    exactly rmhd_imex_step's result (SSP2 and SSP3)."""
    Sim, _, _ = mods
    for scheme in (0, 1):
        wl = WL.khi(n=40, ny=32, seed=5)
        a = Sim.from_workload(wl, scheme=scheme)
        b = Sim.from_workload(wl, scheme=scheme)
        a.step(wl.dt, 3)
        t = C.c_double()
        for _ in range(3):
            for p in range(6 if scheme else 4):
                assert b.lib.rmhd_step_phase(b.h, wl.dt, p, C.byref(t)) == 0
        b.check()
        assert np.array_equal(a.get_state(), b.get_state())
        assert abs(t.value - 3 * wl.dt) < 1e-15


def test_decomposition_refusals(mods):
    Sim, slabs, L = mods
    lib = L.load()
    wl = WL.khi(n=32, seed=6)
    dec = slabs.LocalSlabs(wl, [16, 16])
    s = dec.slabs[0]
    # Gauss's law at a slab edge needs the neighbour: set_prims refused
    rc = lib.rmhd_set_prims(s.h, C.c_void_p(wl.prims[:, :16].copy().ctypes.data), 0)
    assert rc == -5
    dec.set_state(Sim.from_workload(wl).get_state())
    # a slab with neighbours steps only phase by phase
    assert lib.rmhd_imex_step(s.h, wl.dt, 1, None) == -5
    # phases in order
    assert lib.rmhd_step_phase(s.h, wl.dt, 1, None) == -5
    assert lib.rmhd_step_phase(s.h, wl.dt, 0, None) == 0
    assert lib.rmhd_step_phase(s.h, 2 * wl.dt, 1, None) == -1  # one dt per step
    # no adjoint for slabs
    n = C.c_size_t()
    assert lib.rmhd_recording_bytes(s.h, 2, 1, C.byref(n)) == -5
    # halo calls need a slab context; slabs need at least two rows and a 2-D grid
    g = Sim.from_workload(wl)
    assert lib.rmhd_halo_pack(g.h, None, None) == -5
    assert lib.rmhd_halo_doubles(g.h, C.byref(n)) == -5
    cfg = g.cfg
    assert lib.rmhd_slab_workspace_bytes(C.byref(cfg), 0, 1, C.byref(n)) == -1
    assert lib.rmhd_slab_workspace_bytes(C.byref(cfg), 30, 4, C.byref(n)) == -1
    assert lib.rmhd_slab_workspace_bytes(C.byref(cfg), 30, 2, C.byref(n)) == 0
