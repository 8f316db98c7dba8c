"""ctypes wrapper of the FP64 CPU oracle (``rmhd_oracle.c``).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package. It shares nothing with
the CUDA library in ``paper_1808_09721_gb300``; the two are compared element
by element on the same seeded primitive inputs.

The oracle follows Wright & Hawke (arXiv:1808.09721): Sec. 2.1 (models,
primitive recovery), Sec. 2.2.1 + Table 1 (SSP2(222) IMEX), Sec. 2.2.2 (LF flux
splitting + WENO3), Appendix A (two-fluid flux and source).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmhd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODEL_SF, MODEL_TF = 0, 1
BC_OUTFLOW, BC_PERIODIC = 0, 1
NC = {MODEL_SF: 14, MODEL_TF: 18}
NW = {MODEL_SF: 5, MODEL_TF: 10}
NP = {MODEL_SF: 11, MODEL_TF: 16}
GAMMA_SSP2 = 1.0 - 1.0 / np.sqrt(2.0)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("model", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double), ("ymax", C.c_double),
                ("gamma", C.c_double), ("sigma", C.c_double), ("mu_e", C.c_double), ("mu_p", C.c_double),
                ("kappa", C.c_double), ("bc_x", C.c_int), ("bc_y", C.c_int), ("scheme", C.c_int),
                ("nz", C.c_int), ("zmin", C.c_double), ("zmax", C.c_double), ("bc_z", C.c_int)]


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = declare(C.CDLL(build()))
    return _lib


def declare(L):
    """ctypes signatures of the oracle's exported functions on a loaded library
    (the plain build, or the op-counting build of ``oracle/opcount.py``)."""
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(_Cfg)]
    L.orc_destroy.argtypes = [C.c_void_p]
    for name in ("orc_set_prims", "orc_set_cons", "orc_get_cons", "orc_get_prims", "orc_current_L"):
        getattr(L, name).argtypes = [C.c_void_p, _D]
        getattr(L, name).restype = C.c_int
    L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
    L.orc_step.restype = C.c_int
    L.orc_stage_solve.argtypes = [C.c_void_p, C.c_double, _D, _D]
    L.orc_stage_solve.restype = C.c_int
    L.orc_get_padded.argtypes = [C.c_void_p, C.c_int, _D, C.POINTER(C.c_int)]
    L.orc_get_padded.restype = C.c_int
    L.orc_time.argtypes = [C.c_void_p]
    L.orc_time.restype = C.c_double
    L.orc_fail_cell.argtypes = [C.c_void_p]
    L.orc_fail_cell.restype = C.c_int
    L.orc_sf_p2c.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double, _D]
    L.orc_tf_p2c.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _D]
    L.orc_sf_c2p.argtypes = [_D, C.c_double, _D]
    L.orc_tf_c2p.argtypes = [_D, C.c_double, C.c_double, C.c_double, _D]
    L.orc_hydro_c2p.argtypes = [C.c_double, _D, C.c_double, C.c_double, _D]
    L.orc_sf_flux.argtypes = [_D, _D, C.c_double, C.c_double, C.c_int, _D]
    L.orc_sf_flux.restype = None
    L.orc_tf_flux.argtypes = [_D, _D, C.c_double, C.c_double, C.c_double, C.c_int, _D]
    L.orc_tf_flux.restype = None
    L.orc_sf_source.argtypes = [_D, _D, C.c_double, C.c_double, _D]
    L.orc_sf_source.restype = None
    L.orc_tf_source.argtypes = [_D, _D, C.c_double, C.c_double, C.c_double, C.c_double, _D]
    L.orc_tf_source.restype = None
    L.orc_sf_current.argtypes = [_D, _D, C.c_double, _D]
    L.orc_sf_current.restype = None
    L.orc_sf_implicit.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double, _D, _D]
    L.orc_tf_implicit.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, _D, _D]
    L.orc_weno3.argtypes = [C.c_double, C.c_double, C.c_double]
    L.orc_weno3.restype = C.c_double
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_threads.restype = None
    L.orc_get_threads.restype = C.c_int
    return L


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _vec(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


class OracleError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"oracle status {code} {msg}")
        self.code = code


# ---------------------------------------------------------------- per-cell pieces
def sf_p2c(prim11, varrho=0.0, psi=0.0, phi=0.0, gamma=2.0):
    q = np.zeros(14)
    st = lib().orc_sf_p2c(_p(_vec(prim11, 11)), varrho, psi, phi, gamma, _p(q))
    if st:
        raise OracleError(st, "sf_p2c")
    return q


def tf_p2c(prim16, gamma, mu_e, mu_p, psi=0.0, phi=0.0):
    q = np.zeros(18)
    st = lib().orc_tf_p2c(_p(_vec(prim16, 16)), psi, phi, gamma, mu_e, mu_p, _p(q))
    if st:
        raise OracleError(st, "tf_p2c")
    return q


def sf_c2p(q14, gamma):
    w = np.zeros(5)
    st = lib().orc_sf_c2p(_p(_vec(q14, 14)), gamma, _p(w))
    if st:
        raise OracleError(st, "sf_c2p")
    return w


def tf_c2p(q18, gamma, mu_e, mu_p):
    w = np.zeros(10)
    st = lib().orc_tf_c2p(_p(_vec(q18, 18)), gamma, mu_e, mu_p, _p(w))
    if st:
        raise OracleError(st, "tf_c2p")
    return w


def hydro_c2p(D, St, taut, gamma):
    w = np.zeros(5)
    st = lib().orc_hydro_c2p(D, _p(_vec(St, 3)), taut, gamma, _p(w))
    if st:
        raise OracleError(st, "hydro_c2p")
    return w


def sf_flux(q14, w5, gamma, sigma, k):
    f = np.zeros(14)
    lib().orc_sf_flux(_p(_vec(q14, 14)), _p(_vec(w5, 5)), gamma, sigma, k, _p(f))
    return f


def tf_flux(q18, w10, gamma, mu_e, mu_p, k):
    f = np.zeros(18)
    lib().orc_tf_flux(_p(_vec(q18, 18)), _p(_vec(w10, 10)), gamma, mu_e, mu_p, k, _p(f))
    return f


def sf_source(q14, w5, sigma, kappa=1.0):
    s = np.zeros(14)
    lib().orc_sf_source(_p(_vec(q14, 14)), _p(_vec(w5, 5)), sigma, kappa, _p(s))
    return s


def tf_source(q18, w10, sigma, mu_e, mu_p, kappa=1.0):
    s = np.zeros(18)
    lib().orc_tf_source(_p(_vec(q18, 18)), _p(_vec(w10, 10)), sigma, kappa, mu_e, mu_p, _p(s))
    return s


def sf_current(q14, w5, sigma):
    J = np.zeros(3)
    lib().orc_sf_current(_p(_vec(q14, 14)), _p(_vec(w5, 5)), sigma, _p(J))
    return J


def sf_implicit(r14, adt, gamma, sigma, kappa=1.0):
    q, w = np.zeros(14), np.zeros(5)
    st = lib().orc_sf_implicit(_p(_vec(r14, 14)), adt, gamma, sigma, kappa, _p(q), _p(w))
    if st:
        raise OracleError(st, "sf_implicit")
    return q, w


def tf_implicit(r18, adt, gamma, sigma, mu_e, mu_p, kappa=1.0):
    q, w = np.zeros(18), np.zeros(10)
    st = lib().orc_tf_implicit(_p(_vec(r18, 18)), adt, gamma, sigma, kappa, mu_e, mu_p, _p(q), _p(w))
    if st:
        raise OracleError(st, "tf_implicit")
    return q, w


def weno3(fm, f0, fp):
    return lib().orc_weno3(fm, f0, fp)


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ---------------------------------------------------------------- grid simulation
class Sim:
    """A grid run of the oracle: SSP2(222) (scheme 0, Table 1) or SSP3(332)
    (scheme 1, Table 2) IMEX steps with WENO3/LF fluxes."""

    def __init__(self, model, nx, ny, xlim, ylim, gamma, sigma, bc_x, bc_y,
                 mu_e=-1.0, mu_p=1.0, kappa=1.0, scheme=0, nz=1, zlim=(0.0, 1.0), bc_z=1):
        """nz > 1 makes a 3-D grid (needs ny > 1); arrays are then [var][nz][ny][nx]."""
        self.model, self.nx, self.ny, self.nz = model, nx, ny, max(1, nz)
        self.cfg = _Cfg(model, nx, ny, xlim[0], xlim[1], ylim[0], ylim[1], gamma, sigma,
                        mu_e, mu_p, kappa, bc_x, bc_y, scheme, self.nz, zlim[0], zlim[1], bc_z)
        self.h = lib().orc_create(C.byref(self.cfg))
        if not self.h:
            raise OracleError(-1, "orc_create")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    @property
    def nc(self):
        return NC[self.model]

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.nz > 1 else (self.ny, self.nx)

    def _check(self, st, what):
        if st:
            raise OracleError(st, f"{what} (first failing cell {lib().orc_fail_cell(self.h)})")

    def set_prims(self, prims):
        a = _vec(prims)
        assert a.size == NP[self.model] * self.nx * self.ny * self.nz
        self._check(lib().orc_set_prims(self.h, _p(a)), "set_prims")

    def set_cons(self, cons):
        a = _vec(cons)
        assert a.size == self.nc * self.nx * self.ny * self.nz
        self._check(lib().orc_set_cons(self.h, _p(a)), "set_cons")

    def step(self, dt, nsteps=1):
        self._check(lib().orc_step(self.h, dt, nsteps), "step")

    def cons(self):
        out = np.zeros((self.nc,) + self.shape)
        lib().orc_get_cons(self.h, _p(out))
        return out

    def prims(self):
        out = np.zeros((NP[self.model],) + self.shape)
        lib().orc_get_prims(self.h, _p(out))
        return out

    def flux_divergence(self):
        out = np.zeros((self.nc,) + self.shape)
        lib().orc_current_L(self.h, _p(out))
        return out

    def stage_solve(self, adt):
        q = np.zeros((self.nc,) + self.shape)
        w = np.zeros((NW[self.model],) + self.shape)
        self._check(lib().orc_stage_solve(self.h, adt, _p(q), _p(w)), "stage_solve")
        return q, w

    def padded(self, which="cons"):
        """The padded array with its ghost cells: [var][NZ][NY][NX] (NZ = 1 for
        1-D and 2-D grids; 2 ghost layers per side in every active direction)."""
        dims = (C.c_int * 3)()
        w = 0 if which == "cons" else 1
        lib().orc_get_padded(self.h, w, None, dims)
        nv = self.nc if w == 0 else NW[self.model]
        out = np.zeros((nv, dims[2], dims[1], dims[0]))
        lib().orc_get_padded(self.h, w, _p(out), dims)
        return out

    @property
    def t(self):
        return lib().orc_time(self.h)
