"""FP64 operation counts of the method, from the op-counting build of the oracle.

TEST INFRASTRUCTURE. ``opcount.cpp`` compiles ``rmhd_oracle.c`` unchanged with
a counting scalar type (every +, -, x, / and sqrt counts one; see its header),
so the counts below are those of the oracle's own arithmetic.

The oracle is written for checking, not for speed: its flux divergence
re-evaluates each neighbour's flux for every cell (5 per cell and direction)
and each face's reconstruction for both adjacent cells. The *algorithmic*
count of a flux pass therefore composes the counted pieces with the
multiplicities the method needs (Sec. 2.2.2 and Eq. implicit stage /
correction stage):

  per cell and direction   one physical flux f(q, w) (Eq. resistive RMHD or
                           Appendix A), the splitting f+- = (f +- q)/2 of
                           every component (4 ops), and the face difference
                           -(F_{i+1/2} - F_{i-1/2})/dx accumulated into L
                           (3 ops per component; 2 in the first direction,
                           whose accumulation starts from zero);
  per face and component   two WENO3 reconstructions and their sum (one face
                           per cell and direction on a periodic grid);
  per cell                 one source evaluation Psi(q, w);
  per cell and output      base + c_L L for every component (2 ops) and + c_Psi Psi
                           for every component with a source (2 ops).

Trivial operations (a product with an exact 0 or +-1, a sum with an exact 0)
are not counted (``opcount.cpp``): the oracle writes cross products and the B
and E fluxes as full Levi-Civita sums, of which only the nonzero terms are
arithmetic. The pieces are counted on generic cells (no exact zeros or unit
values in the data), so every counted operation is one the method needs.

The stage solve and the whole step are reported as the oracle executes them
(forward-difference Jacobians, Newton iterated to a round-off fixed point):
those are the oracle's counts, not a minimal count of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import _Cfg, declare

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opcount.cpp")
_ORC = os.path.join(_HERE, "rmhd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_count.so")
_D = C.POINTER(C.c_double)
_lib = None

# operation classes counted by the build, in the order orc_count_get writes them
KINDS = ("add", "sub", "mul", "div", "sqrt")


def build(force: bool = False) -> str:
    """Compile the counting build with g++ (no OpenMP, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_ORC))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cmd = ["g++", "-std=c++17", "-O2", "-fpermissive", "-w", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = declare(C.CDLL(build()))
        L.orc_count_reset.argtypes = []
        L.orc_count_reset.restype = None
        L.orc_count_get.argtypes = [C.POINTER(C.c_longlong)]
        L.orc_count_get.restype = None
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def count(fn) -> dict:
    """Operations executed by fn() in the counting build: {kind: n, 'total': n}."""
    L = lib()
    L.orc_count_reset()
    fn()
    out = (C.c_longlong * 5)()
    L.orc_count_get(out)
    d = {k: int(out[i]) for i, k in enumerate(KINDS)}
    d["total"] = sum(d[k] for k in KINDS)
    return d


def _sf_cell(seed=0):
    """A generic admissible single-fluid cell: every component nonzero."""
    rng = np.random.default_rng(seed)
    q = np.ascontiguousarray(rng.uniform(0.5, 1.5, 14))
    w = np.array([1.1, 0.21, -0.13, 0.17, 0.9])  # rho, v, p
    return q, w


def _tf_cell(seed=0):
    rng = np.random.default_rng(seed)
    q = np.ascontiguousarray(rng.uniform(0.5, 1.5, 18))
    w = np.array([0.5, 0.21, -0.13, 0.17, 0.45, 0.55, -0.11, 0.12, -0.09, 0.5])
    return q, w


def pieces(model: int) -> dict:
    """Counted operations of one call of each piece of the flux pass."""
    L = lib()
    out = np.zeros(18)
    if model == 0:
        q, w = _sf_cell()
        flux = count(lambda: L.orc_sf_flux(_p(q), _p(w), 4.0 / 3.0, 1e3, 0, _p(out)))
        src = count(lambda: L.orc_sf_source(_p(q), _p(w), 1e3, 1.0, _p(out)))
        nc, ns = 14, 5
    else:
        q, w = _tf_cell()
        flux = count(lambda: L.orc_tf_flux(_p(q), _p(w), 4.0 / 3.0, -1e3, 1e3, 0, _p(out)))
        src = count(lambda: L.orc_tf_source(_p(q), _p(w), 1e4, 1.0, -1e3, 1e3, _p(out)))
        nc, ns = 18, 9
    weno = count(lambda: L.orc_weno3(0.3, 0.7, -0.2))
    return {"flux": flux["total"], "source": src["total"], "weno3": weno["total"], "nc": nc, "ns": ns}


def flux_pass_ops(model: int, ndim: int, nout: int) -> int:
    """Algorithmic FP64 operations per interior cell of one flux pass with
    `nout` stage combinations, on a periodic grid (composition in the module
    docstring)."""
    pc = pieces(model)
    nc, ns = pc["nc"], pc["ns"]
    per_dir = pc["flux"] + nc * 4 + nc * (2 * pc["weno3"] + 1) + nc * 3
    return ndim * per_dir - nc + pc["source"] + nout * (2 * nc + 2 * ns)


def _sim(wl, cons=None):
    """A counting-build run of workload wl, from its primitives or, if given,
    from the conserved state `cons`."""
    L = lib()
    cfg = _Cfg(wl.model, wl.nx, wl.ny, wl.xlim[0], wl.xlim[1], wl.ylim[0], wl.ylim[1], wl.gamma, wl.sigma,
               wl.mu_e, wl.mu_p, wl.kappa, wl.bc_x, wl.bc_y, 0, 1, 0.0, 1.0, 1)
    h = L.orc_create(C.byref(cfg))
    if cons is None:
        prims = np.ascontiguousarray(wl.prims, dtype=np.float64)
        assert L.orc_set_prims(h, _p(prims)) == 0
    else:
        assert L.orc_set_cons(h, _p(np.ascontiguousarray(cons, dtype=np.float64))) == 0
    return L, h


def oracle_step_ops(wl, what: str = "step", cons=None) -> float:
    """Operations per interior cell the oracle itself executes on workload wl
    (from its primitives, or from the conserved state `cons`): what = 'step'
    (one SSP2(222) step), 'stage' (the stage-1 implicit solve) or 'divergence'
    (one flux divergence L(q), with the oracle's redundancy)."""
    L, h = _sim(wl, cons)
    try:
        n = wl.nx * wl.ny
        if what == "step":
            c = count(lambda: L.orc_step(h, wl.dt, 1))
        elif what == "stage":
            q = np.zeros((wl.prims.shape[0] + 8) * n)
            wv = np.zeros(10 * n)
            g = 1.0 - 1.0 / np.sqrt(2.0)
            c = count(lambda: L.orc_stage_solve(h, g * wl.dt, _p(q), _p(wv)))
        else:
            out = np.zeros(18 * n)
            c = count(lambda: L.orc_current_L(h, _p(out)))
        return c["total"] / n
    finally:
        L.orc_destroy(h)


def table() -> dict:
    """The counts quoted next to the measured kernel times (per interior cell)."""
    from paper_1808_09721_gb300 import workloads as WL
    khi = WL.khi(n=64, seed=0)
    tfs = WL.tf_sheet(n=32, seed=1)
    return {
        "pieces_sf": pieces(0), "pieces_tf": pieces(1),
        "sf_2d_flux1": flux_pass_ops(0, 2, 2), "sf_2d_flux2": flux_pass_ops(0, 2, 1),
        "tf_2d_flux1": flux_pass_ops(1, 2, 2), "tf_2d_flux2": flux_pass_ops(1, 2, 1),
        "oracle_khi64_stage": oracle_step_ops(khi, "stage"),
        "oracle_khi64_step": oracle_step_ops(khi, "step"),
        "oracle_tf32_stage": oracle_step_ops(tfs, "stage"),
    }


if __name__ == "__main__":
    import json
    print(json.dumps(table(), indent=1))
