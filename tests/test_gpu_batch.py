"""Batched ensemble of independent 1-D runs (one context, packed state,
persistent kernels over a (run, tile) work list, one CUDA graph per step):
every run against the FP64 oracle run on its own with its own CFL time step."""
import numpy as np
import pytest

import oracle as O
from conftest import parity_errors, parity_scale
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


def _runs():
    runs = WL.batch_tubes(count=7, seed=11, nmin=60, nmax=400)
    runs.append(WL.batch_tubes(count=1, seed=12, nmin=3, nmax=3)[0])     # smaller than a stencil
    runs.append(WL.batch_tubes(count=1, seed=13, nmin=129, nmax=129)[0]) # ragged last tile
    return runs


def _oracle(wl, steps):
    o = O.Sim(wl.model, wl.nx, 1, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    o.set_prims(wl.prims)
    o.step(wl.dt, steps)
    return o.cons()


def test_batch_fp64_matches_oracle_per_run(Sim):
    runs = _runs()
    b = Sim.batch(runs)
    b.step(0.0, 8)   # each run with its own dt = cfl * dx
    b.check()
    got = b.unpack(b.cons())
    for wl, g in zip(runs, got):
        err = parity_errors(0, g, _oracle(wl, 8))
        assert np.all(err <= 1e-9), (wl.name, wl.nx, wl.sigma, err)


def test_batch_mixed_matches_oracle_per_run(Sim):
    runs = _runs()
    b = Sim.batch(runs, precision=1)
    b.step(0.0, 8)
    b.check()
    got = b.unpack(b.cons())
    for wl, g in zip(runs, got):
        want = _oracle(wl, 8)
        l1 = np.abs(g - want).reshape(14, -1).mean(axis=1) / parity_scale(0, want)
        assert np.all(l1 <= 1e-4), (wl.name, l1)


def test_autotune_keeps_state_and_results(Sim):
    runs = WL.batch_tubes(count=24, seed=14, nmin=100, nmax=900)
    a = Sim.batch(runs, precision=1)
    b = Sim.batch(runs, precision=1)
    before = b.cons()
    choice = b.autotune()
    assert choice["tile_x"] in (64, 128, 256) and choice["flux_ctas"] >= 1 and choice["stage_threads"] in (64, 128, 256)
    np.testing.assert_array_equal(b.cons(), before)
    a.step(0.0, 5)
    b.step(0.0, 5)
    a.check()
    b.check()
    # the tile width only changes which CTA computes a cell, not its arithmetic
    np.testing.assert_array_equal(a.cons(), b.cons())


def _sampled(runs):
    """Tubes checked against the oracle: the first and last, the one with the
    coldest dense right state near the initial jump (215), the stiffest and
    the longest."""
    sig = int(np.argmax([w.sigma for w in runs]))
    big = int(np.argmax([w.nx for w in runs]))
    return sorted({0, 215, len(runs) - 1, sig, big})


def test_full_512_tube_configuration_mixed(Sim):
    """The benchmark's 512-tube ensemble (N up to 4096, sigma up to 1e6, density
    and pressure ratios up to 100), its whole 400-step run in the mixed form:
    no solver failure anywhere, and the sampled tubes match the oracle."""
    runs = WL.batch_tubes(count=512, seed=2)
    b = Sim.batch(runs, precision=1)
    b.step(0.0, 400)
    b.check()
    got = b.unpack(b.cons())
    for r in _sampled(runs):
        want = _oracle(runs[r], 400)
        l1 = np.abs(got[r] - want).reshape(14, -1).mean(axis=1) / parity_scale(0, want)
        assert np.all(l1 <= 1e-4), (r, l1)


def test_full_512_tube_configuration_fp64(Sim):
    """The same 400-step run in the FP64 form: sampled tubes within 1e-9."""
    runs = WL.batch_tubes(count=512, seed=2)
    b = Sim.batch(runs)
    b.step(0.0, 400)
    b.check()
    got = b.unpack(b.cons())
    for r in _sampled(runs):
        err = parity_errors(0, got[r], _oracle(runs[r], 400))
        assert np.all(err <= 1e-9), (r, runs[r].nx, runs[r].sigma, err)
