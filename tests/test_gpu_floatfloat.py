"""Float-float flux form (RMHD_FLOATFLOAT) against the FP64 CPU oracle.

The WENO3 / flux arithmetic runs in float-float (pairs of FP32 numbers, about
48 significant bits) on the FP32 pipes; sources, current, update and the
implicit stage solves stay FP64. The bar is the FP64 one: relative L-infinity
<= 1e-9 per conserved variable (conftest.parity_scale), on the same cases as
the FP64 parity tests -- 1-D shocks and stiff tubes, 2-D periodic and outflow
grids, SSP3(332), 3-D, and the 1024^2 benchmark grid on sampled cells -- plus
agreement with the GPU's own FP64 form to 1e-11; the two-fluid model on the
current sheet (2-D) and the pair / electron-proton Brio-Wu tubes. Batches and
the adjoint refuse the mode."""
import numpy as np
import pytest

import oracle as O
from conftest import parity_errors, parity_scale
from paper_1808_09721_gb300 import RmhdError
from paper_1808_09721_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-9
FF = 2


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


def oracle_run(wl, nsteps, scheme=0):
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p, kappa=wl.kappa, scheme=scheme, nz=wl.nz, zlim=wl.zlim, bc_z=wl.bc_z)
    o.set_prims(wl.prims)
    o.step(wl.dt, nsteps)
    return o.cons()


def gpu_run(Sim, wl, nsteps, precision=FF, scheme=0):
    g = Sim.from_workload(wl, precision=precision, scheme=scheme)
    g.step(wl.dt, nsteps)
    g.check()
    return g.cons()


def err(got, want):
    return parity_errors(0, got.reshape(14, -1, 1), want.reshape(14, -1, 1))


def err_tf(got, want, wl):
    return parity_errors(1, got, want, max(abs(wl.mu_e), abs(wl.mu_p)))


@pytest.mark.parametrize("name,make,steps,scheme", [
    ("brio_wu_full", lambda: WL.brio_wu(), 400, 0),
    ("khi_64", lambda: WL.khi(n=64, seed=0), 6, 0),
    ("khi_70x45", lambda: WL.khi(n=70, ny=45, seed=2), 4, 0),
    ("field_loop_32", lambda: WL.field_loop(n=32), 5, 0),
    ("khi_48_ssp3", lambda: WL.khi(n=48, seed=1), 4, 1),
    ("khi3d_12", lambda: WL.khi3d(n=12, seed=4), 3, 0),
])
def test_floatfloat_parity(Sim, name, make, steps, scheme):
    wl = make()
    e = err(gpu_run(Sim, wl, steps, scheme=scheme), oracle_run(wl, steps, scheme))
    assert np.all(e <= TOL), e


def test_floatfloat_stiff_tubes_and_outflow(Sim):
    for wl in WL.batch_tubes(count=4, seed=5, nmin=100, nmax=300):
        e = err(gpu_run(Sim, wl, 20), oracle_run(wl, 20))
        assert np.all(e <= TOL), (wl.name, wl.sigma, e)
    wl = WL.khi(n=20, ny=12, seed=7)
    wl = wl.with_prims(wl.prims, bc_x=WL.OUTFLOW, bc_y=WL.OUTFLOW)
    assert np.all(err(gpu_run(Sim, wl, 3), oracle_run(wl, 3)) <= TOL)
    for nx in (1, 2, 3):
        wl = WL.brio_wu(nx=nx)
        assert np.all(err(gpu_run(Sim, wl, 3), oracle_run(wl, 3)) <= TOL)


def test_floatfloat_long_tube_agrees_with_fp64(Sim):
    """A 1-D grid above 4864 cells takes the 128-cell tile (its own kernel
    instantiation): 50 steps of a 6000-cell Brio-Wu tube against the FP64 form."""
    wl = WL.brio_wu(nx=6000)
    a = gpu_run(Sim, wl, 50, precision=0)
    b = gpu_run(Sim, wl, 50)
    assert np.all(err(b, a) <= 1e-11), err(b, a)


def test_floatfloat_full_size_khi(Sim):
    """The 1024^2 benchmark grid: one step against the GPU's FP64 form on every
    cell (<= 1e-11), and sampled cells against the oracle on 16 x 16 periodic
    windows (a cell after one step depends only on cells within 4 of it)."""
    wl = WL.khi(n=1024, seed=0)
    n = wl.nx
    got = gpu_run(Sim, wl, 1)
    ref = gpu_run(Sim, wl, 1, precision=0)
    assert np.all(err(got, ref) <= 1e-11), err(got, ref)
    scale = parity_scale(0, got)
    rng = np.random.default_rng(39)
    h = 8
    for _ in range(4):
        j0, i0 = (int(x) for x in rng.integers(0, n, size=2))
        jj, ii = np.arange(j0 - h, j0 + h) % n, np.arange(i0 - h, i0 + h) % n
        win = np.ascontiguousarray(wl.prims[:, jj][:, :, ii])
        sub = wl.with_prims(win, nx=2 * h, ny=2 * h, bc_x=WL.OUTFLOW, bc_y=WL.OUTFLOW,
                            xlim=(0.0, 2 * h * wl.dx), ylim=(0.0, 2 * h * wl.dy))
        want = oracle_run(sub, 1)[:, h, h]
        assert np.all(np.abs(got[:, j0, i0] - want) <= TOL * scale), (j0, i0)


@pytest.mark.parametrize("name,make,steps", [
    ("tf_sheet_40", lambda: WL.tf_sheet(n=40, seed=2), 4),
    ("tf_brio_wu_pair", lambda: WL.tf_brio_wu(nx=400), None),
    ("tf_brio_wu_ep", lambda: WL.tf_brio_wu(nx=200, mass_ratio=100.0), None),
])
def test_floatfloat_two_fluid_parity(Sim, name, make, steps):
    wl = make()
    steps = wl.nsteps if steps is None else steps
    e = err_tf(gpu_run(Sim, wl, steps), oracle_run(wl, steps), wl)
    assert np.all(e <= TOL), e


def test_floatfloat_two_fluid_512_agrees_with_fp64(Sim):
    """The two-fluid sheet 512^2 the bench times: 2 steps against the FP64 form."""
    wl = WL.tf_sheet(n=512, seed=1)
    e = err_tf(gpu_run(Sim, wl, 2), gpu_run(Sim, wl, 2, precision=0), wl)
    assert np.all(e <= 1e-11), e


def test_floatfloat_scope_is_refused(Sim):
    with pytest.raises(RmhdError):
        Sim.batch(WL.batch_tubes(count=2, seed=3, nmin=40, nmax=60), precision=FF)
    wl = WL.field_loop(n=16)
    g = Sim.from_workload(wl, precision=FF)
    with pytest.raises(RmhdError):
        g.record(2, 1)
