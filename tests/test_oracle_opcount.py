"""The op-counting build of the oracle (oracle/opcount.cpp, oracle/opcount.py):
it computes exactly what the plain oracle computes, its counter counts what a
hand count of the written formulas gives, and the algorithmic FP64 operation
counts quoted by bench.py are the ones it produces.

Paper: Wright & Hawke, arXiv:1808.09721 -- Sec. 2.2.2 (WENO3 reconstruction,
Lax-Friedrichs splitting), Sec. 2.1.1 (Ohm's law), Table 1 (SSP2(222)).
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle as O
from oracle import opcount as OC
from paper_1808_09721_gb300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counting_build_is_bitwise_the_oracle():
    """One SSP2(222) step of a KHI window and of a two-fluid sheet: the counting
    build's state equals the plain build's bit for bit (same operations, same
    order; the counter does not change any result)."""
    for wl in (WL.khi(n=20, ny=12, seed=3), WL.tf_sheet(n=10, seed=2)):
        plain = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
                      mu_e=wl.mu_e, mu_p=wl.mu_p)
        O.set_threads(1)
        plain.set_prims(wl.prims)
        plain.step(wl.dt, 1)
        want = plain.cons()
        L, h = OC._sim(wl)
        try:
            assert L.orc_step(h, wl.dt, 1) == 0
            got = np.zeros_like(want)
            L.orc_get_cons(h, OC._p(got))
        finally:
            L.orc_destroy(h)
        assert np.array_equal(got, want)


def test_counter_matches_hand_counts():
    """WENO3 as the oracle writes it (Sec. 2.2.2): p0 = -f_m/2 + 3 f_0/2 (2 mul, 1 add),
    p1 = f_0/2 + f_p/2 (3), beta0 = (f_0 - f_m)(f_0 - f_m) (2 sub, 1 mul), beta1 (3),
    alpha_k = d_k/((eps + beta_k)(eps + beta_k)) (2 add, 1 mul, 1 div, each), and
    (alpha0 p0 + alpha1 p1)/(alpha0 + alpha1) (2 mul, 2 add, 1 div): 25.
    Ohm's current (Sec. 2.1.1) on a generic cell: W = 1/sqrt(1 - v.v) (3 mul,
    2 add, 1 sub, 1 sqrt, 1 div), v x B (6 mul, 3 sub), v.E (3 mul, 2 add), and
    per component varrho v_i + W sigma (E_i + (v x B)_i - (v.E) v_i) (4 mul,
    3 add/sub): 8 + 9 + 5 + 21 = 43."""
    c = OC.count(lambda: OC.lib().orc_weno3(0.3, 0.7, -0.2))
    assert c["total"] == 25 and c["div"] == 3 and c["mul"] == 10 and c["sub"] == 4
    q, w = OC._sf_cell()
    J = np.zeros(3)
    c = OC.count(lambda: OC.lib().orc_sf_current(OC._p(q), OC._p(w), 10.0, OC._p(J)))
    assert c["total"] == 43 and c["sqrt"] == 1 and c["div"] == 1
    # a product with an exact 1 or 0 is not arithmetic: W sigma with sigma = 1 counts one less
    c1 = OC.count(lambda: OC.lib().orc_sf_current(OC._p(q), OC._p(w), 1.0, OC._p(J)))
    assert c1["total"] == 40


def _bench_constants():
    spec = importlib.util.spec_from_file_location("bench_consts", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.ALG_FP64_FLOPS_PER_CELL


def test_bench_quotes_the_counted_algorithmic_operations():
    consts = _bench_constants()
    assert consts["flux1"] == OC.flux_pass_ops(0, 2, 2)
    assert consts["flux2"] == OC.flux_pass_ops(0, 2, 1)
    assert consts["tf_flux1"] == OC.flux_pass_ops(1, 2, 2)
    assert consts["tf_flux2"] == OC.flux_pass_ops(1, 2, 1)


@pytest.mark.parametrize("model", [0, 1])
def test_flux_pass_composition_matches_the_oracle_divergence(model):
    """The oracle's flux divergence evaluates 5 neighbour fluxes per cell and
    direction and 4 WENO3 reconstructions per component (both faces of the
    cell); with those multiplicities the composed per-piece count reproduces
    the counted divergence exactly (periodic 2-D grid, generic data), which
    checks the composition's terms."""
    pc = OC.pieces(model)
    wl = WL.khi(n=16, ny=12, seed=1) if model == 0 else WL.tf_sheet(n=12, seed=1)
    nc = pc["nc"]
    # generic data: no exact zeros or unit values (the workload has v_z = 0,
    # psi = phi = 0, ...), made by perturbing every conserved variable
    o = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
              mu_e=wl.mu_e, mu_p=wl.mu_p)
    o.set_prims(wl.prims)
    q = o.cons()
    rng = np.random.default_rng(5)
    q += 1e-4 * rng.uniform(0.5, 1.0, q.shape) * np.maximum(np.abs(q).max(axis=(1, 2), keepdims=True), 1e-3)
    per_dir = 5 * (pc["flux"] + 4 * nc) + nc * (4 * pc["weno3"] + 2 + 3)
    redundant = 2 * per_dir - nc  # the first direction's accumulation starts from zero
    got = OC.oracle_step_ops(wl, "divergence", cons=q)
    assert got == redundant
    # the algorithmic pass: one flux per cell and direction, one pair of
    # reconstructions per face, plus the source and the stage combinations
    alg = 2 * (pc["flux"] + 4 * nc + nc * (2 * pc["weno3"] + 1) + 3 * nc) - nc + pc["source"] + \
        2 * (2 * nc + 2 * pc["ns"])
    assert OC.flux_pass_ops(model, 2, 2) == alg
