"""The state and primitive calls through the three kinds of caller memory.

Device arrays and page-locked host arrays are read and written in place by
the library's kernels (host arrays over the host-GPU link); pageable host
arrays go through the staging buffer. All three must give bitwise the same
results, on single grids of both models and on a batched ensemble, for the
fused recovery + output of rmhd_get_prims after a step as well as for the
plain output of fresh primitives. A RMHD_DEVICE pointer that is host memory is
refused before any kernel runs."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


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


def pinned(shape):
    import torch
    a = torch.empty(int(np.prod(shape)), dtype=torch.float64, pin_memory=True).numpy().reshape(shape)
    a[...] = np.nan
    return a


def device(shape):
    import torch
    return torch.full((int(np.prod(shape)),), float("nan"), dtype=torch.float64, device="cuda")


def outputs(sim, kind, call, nvar):
    """Run an output call (prims / cons / get_state) into a buffer of `kind`."""
    shape = (nvar,) + sim.shape
    if kind == "pageable":
        buf = np.full(shape, np.nan)
    elif kind == "pinned":
        buf = pinned(shape)
    else:
        buf = device(shape)
    getattr(sim, call)(out=buf)
    return np.array(buf.cpu().numpy().reshape(shape) if kind == "device" else buf)


def input_of(kind, arr):
    if kind == "pageable":
        return np.ascontiguousarray(arr)
    if kind == "pinned":
        p = pinned(arr.shape)
        p[...] = arr
        return p
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr).ravel()).cuda()


CASES = [
    ("khi", lambda: WL.khi(n=40, seed=5)),
    ("tf_sheet", lambda: WL.tf_sheet(n=20, seed=6)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_set_prims_and_outputs_agree_across_memory_kinds(Sim, name, make):
    wl = make()
    kinds = ("pageable", "pinned", "device")
    sims = {}
    for k in kinds:
        s = Sim.from_workload(wl)        # constructor uploads from pageable memory
        s.set_prims(input_of(k, wl.prims))
        sims[k] = s
    ref = outputs(sims["pageable"], "pageable", "cons", sims["pageable"].nc)
    for k in kinds:
        for out_kind in kinds:
            # fresh primitives: the plain output kernel
            np.testing.assert_array_equal(outputs(sims[k], out_kind, "prims", sims[k].np),
                                          outputs(sims["pageable"], "pageable", "prims", sims[k].np))
            np.testing.assert_array_equal(outputs(sims[k], out_kind, "cons", sims[k].nc), ref)
    # after a step the first get_prims recovers and writes in one kernel; later
    # ones write the recovered primitives: every order and kind must agree
    got = {}
    for k in kinds:
        sims[k].step(wl.dt, 2)
        got[k] = outputs(sims[k], k, "prims", sims[k].np)   # fused recovery + output into `k` memory
    for k in kinds:
        np.testing.assert_array_equal(got[k], got["pageable"])
        for out_kind in kinds:
            np.testing.assert_array_equal(outputs(sims[k], out_kind, "prims", sims[k].np), got["pageable"])
    assert np.isfinite(got["pageable"]).all()


@pytest.mark.parametrize("name,make", CASES)
def test_state_round_trip_through_pinned_memory(Sim, name, make):
    wl = make()
    a = Sim.from_workload(wl)
    a.step(wl.dt, 2)
    nstate = a.nc + a.nw
    st_page = outputs(a, "pageable", "get_state", nstate)
    st_pin = outputs(a, "pinned", "get_state", nstate)
    st_dev = outputs(a, "device", "get_state", nstate)
    np.testing.assert_array_equal(st_pin, st_page)
    np.testing.assert_array_equal(st_dev, st_page)
    b = Sim.from_workload(wl)
    b.set_state(input_of("pinned", st_page))
    a.step(wl.dt, 2)
    b.step(wl.dt, 2)
    np.testing.assert_array_equal(outputs(b, "pinned", "cons", b.nc), outputs(a, "pageable", "cons", a.nc))
    c = Sim.from_workload(wl)
    c.set_cons(input_of("pinned", st_page[:a.nc]))
    np.testing.assert_array_equal(outputs(c, "pageable", "cons", c.nc), st_page[:a.nc])


def test_batch_set_prims_from_pinned_memory(Sim):
    runs = WL.batch_tubes(count=5, seed=21, nmin=40, nmax=300)
    a = Sim.batch(runs)
    b = Sim.batch(runs)
    b.set_prims(input_of("pinned", b.pack([w.prims for w in runs])))
    for s in (a, b):
        s.step(0.0, 3)
    np.testing.assert_array_equal(outputs(b, "pinned", "prims", b.np), outputs(a, "pageable", "prims", a.np))


def test_device_flag_on_host_memory_is_refused(Sim):
    from paper_1808_09721_gb300 import _lib as L
    invalid = next(code for code, name in L.ERRORS.items() if name == "RMHD_ERR_INVALID")
    wl = WL.khi(n=16, seed=7)
    s = Sim.from_workload(wl)
    before = outputs(s, "pageable", "cons", s.nc)
    for host in (np.zeros((s.np,) + s.shape), pinned((s.np,) + s.shape)):
        code = s.lib.rmhd_get_prims(s.h, C.c_void_p(host.ctypes.data), L.DEVICE)
        assert code == invalid
        assert "not device memory" in s.lib.rmhd_last_error(s.h).decode()
        code = s.lib.rmhd_set_prims(s.h, C.c_void_p(host.ctypes.data), L.DEVICE)
        assert code == invalid
    np.testing.assert_array_equal(outputs(s, "pageable", "cons", s.nc), before)
