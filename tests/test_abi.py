"""C ABI checks that need no GPU: the library loads, exports every function
include/rmhd.h declares, and validates configurations on the host."""
import ctypes as C
import os
import re

import pytest

from paper_1808_09721_gb300 import _lib as L
from paper_1808_09721_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "rmhd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rmhd_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert sorted(L.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.rmhd_version()


def _cfg(**kw):
    base = dict(model=0, nx=64, ny=32, xmin=0.0, xmax=1.0, ymin=0.0, ymax=0.5, gamma=4 / 3, sigma=1e3,
                mu_e=-1.0, mu_p=1.0, kappa=1.0, cfl=0.4, bc_x=1, bc_y=1, precision=0)
    base.update(kw)
    c = L.Config()
    for k, v in base.items():
        setattr(c, k, v)
    return c


def test_workspace_bytes_and_validation(lib):
    n = C.c_size_t()
    assert lib.rmhd_workspace_bytes(C.byref(_cfg()), C.byref(n)) == 0
    # 6 state arrays of 14/5 planes + staging + small buffers, 256-byte aligned
    plane = (64 * 32 + 63) // 64 * 64 * 8
    assert n.value >= (4 * 14 + 2 * 5) * plane and n.value % 256 == 0
    n2 = C.c_size_t()
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(model=1)), C.byref(n2)) == 0 and n2.value > n.value
    # float-float flux form, both models
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(precision=2)), C.byref(n2)) == 0
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(precision=2, model=1)), C.byref(n2)) == 0
    for bad in (dict(model=7), dict(nx=0), dict(ny=0), dict(gamma=2.5), dict(gamma=1.0), dict(sigma=0.0), dict(bc_x=3),
                dict(precision=3), dict(model=1, mu_e=1.0, mu_p=1.0), dict(xmax=-1.0),
                dict(nx=1, ny=600000)):  # more rows than the flux kernel's grid can hold
        assert lib.rmhd_workspace_bytes(C.byref(_cfg(**bad)), C.byref(n)) == -1, bad


def test_null_arguments_are_rejected(lib):
    assert lib.rmhd_workspace_bytes(None, None) == -1
    assert lib.rmhd_create(None, C.byref(_cfg()), None, None, 0) == -1
    h = C.c_void_p()
    assert lib.rmhd_create(C.byref(h), C.byref(_cfg(nx=-3)), None, None, 0) == -1
    assert not h.value
    assert lib.rmhd_last_error(None) == b"null context"
    lib.rmhd_destroy(None)


def test_batch_workspace_bytes(lib):
    nx = (C.c_int * 3)(100, 4096, 7)
    n = C.c_size_t()
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1)), 3, nx, C.byref(n)) == 0
    total = 100 + 4096 + 7
    plane = (total + 63) // 64 * 64 * 8
    assert n.value >= (4 * 14 + 2 * 5) * plane + total * 4 and n.value % 256 == 0
    bad = (C.c_int * 2)(10, 0)
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1)), 2, bad, C.byref(n)) == -1
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1)), 0, nx, C.byref(n)) == -1
    # batches take the FP64 and mixed forms; the float-float form is single-grid only
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1, precision=1)), 3, nx, C.byref(n)) == 0
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1, precision=2)), 3, nx, C.byref(n)) == -1


def test_scheme_selection(lib):
    """SSP3(332) (scheme 1, Table 2) needs one more 14-plane buffer than
    SSP2(222); other schemes are invalid; batches take SSP2(222) only."""
    n2, n3 = C.c_size_t(), C.c_size_t()
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(scheme=0)), C.byref(n2)) == 0
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(scheme=1)), C.byref(n3)) == 0
    plane = (64 * 32 + 63) // 64 * 64 * 8
    assert n3.value - n2.value == (14 * plane + 255) // 256 * 256
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(scheme=2)), C.byref(n3)) == -1
    nx = (C.c_int * 2)(100, 200)
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1, scheme=1)), 2, nx, C.byref(n3)) == -1
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1, scheme=0)), 2, nx, C.byref(n3)) == 0


def test_3d_configuration(lib):
    """nz > 1: one more N_c-plane buffer (L_x + L_y of a flux pass); needs ny > 1
    and zlen > 0; not for batches."""
    n2, n3 = C.c_size_t(), C.c_size_t()
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(nz=1)), C.byref(n2)) == 0
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(nz=4, zlen=1.0)), C.byref(n3)) == 0
    assert n3.value > 4 * n2.value
    n4 = C.c_size_t()
    assert lib.rmhd_workspace_bytes(C.byref(_cfg(nz=4, zlen=1.0, model=1)), C.byref(n4)) == 0
    for bad in (dict(nz=4, zlen=0.0), dict(nz=4, zlen=1.0, ny=1),
                dict(nz=4, zlen=1.0, bc_z=5), dict(nz=-2),
                dict(nz=70000, zlen=1.0, ny=2, nx=2), dict(nz=2, zlen=1.0, ny=70000, nx=2)):
        assert lib.rmhd_workspace_bytes(C.byref(_cfg(**bad)), C.byref(n3)) == -1, bad
    nx = (C.c_int * 2)(100, 200)
    assert lib.rmhd_batch_workspace_bytes(C.byref(_cfg(ny=1, nz=3, zlen=1.0)), 2, nx, C.byref(n3)) == -1
