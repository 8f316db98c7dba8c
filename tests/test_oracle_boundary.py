"""Pins of the CPU oracle's initial charge density and boundary conditions (no GPU).

Paper: Wright & Hawke, arXiv:1808.09721 -- Sec. 2.1.1: the charge density
varrho is an evolved variable whose initial value follows Gauss's law
div E = varrho (psi = phi = 0 initially); here div E is the second-order
central difference with neighbours taken through the boundary conditions.
Boundary conditions: outflow copies the nearest interior cell into the two
ghost layers, periodic wraps.

The Gauss's-law pins use fields whose central differences have closed forms:
sin(a + h) - sin(a - h) = 2 cos(a) sin(h) and cos(a + h) - cos(a - h) =
-2 sin(a) sin(h), so on a periodic grid the discrete divergence is known
exactly at every cell (a one-sided difference, a missing 1/2 or a wrong
neighbour fails them by O(1)). The outflow pin uses a linear field: interior
cells give exactly the slope, and the boundary cells, whose ghost copies the
cell itself, give half of it. The ghost pins read the padded arrays directly.
"""
import math

import numpy as np
import pytest

import oracle as O

TWO_PI = 2.0 * math.pi


def _sf_prims_with_e(E, shape):
    """rho = 1, v = 0, p = 1, B = 0 and the given E (3 fields of `shape`)."""
    n = int(np.prod(shape))
    P = np.zeros((11,) + tuple(shape))
    P[0] = 1.0
    P[4] = 1.0
    P[8:11] = E
    assert P.size == 11 * n
    return np.ascontiguousarray(P)


def test_gauss_law_periodic_2d_closed_form():
    nx, ny = 16, 12
    dx, dy = 1.0 / nx, 1.0 / ny
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)  # [ny][nx]
    E = np.stack([np.sin(TWO_PI * X), np.cos(TWO_PI * Y), 0.3 * np.ones_like(X)])
    s = O.Sim(O.MODEL_SF, nx, ny, (0, 1), (0, 1), 4.0 / 3.0, 10.0, O.BC_PERIODIC, O.BC_PERIODIC)
    s.set_prims(_sf_prims_with_e(E, (ny, nx)))
    q = s.cons()
    want = np.cos(TWO_PI * X) * math.sin(TWO_PI * dx) / dx - np.sin(TWO_PI * Y) * math.sin(TWO_PI * dy) / dy
    assert np.max(np.abs(q[11] - want)) <= 2e-14 * np.max(np.abs(want))
    # psi = phi = 0 initially (Sec. 2.1.1)
    assert np.all(q[12] == 0.0) and np.all(q[13] == 0.0)


def test_gauss_law_periodic_3d_closed_form():
    nx, ny, nz = 10, 8, 6
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")  # [nz][ny][nx]
    E = np.stack([np.sin(TWO_PI * X), np.cos(TWO_PI * Y), np.sin(TWO_PI * Z)])
    s = O.Sim(O.MODEL_SF, nx, ny, (0, 1), (0, 1), 4.0 / 3.0, 10.0, O.BC_PERIODIC, O.BC_PERIODIC,
              nz=nz, zlim=(0, 1), bc_z=O.BC_PERIODIC)
    s.set_prims(_sf_prims_with_e(E, (nz, ny, nx)))
    q = s.cons()
    want = (np.cos(TWO_PI * X) * math.sin(TWO_PI * dx) / dx - np.sin(TWO_PI * Y) * math.sin(TWO_PI * dy) / dy +
            np.cos(TWO_PI * Z) * math.sin(TWO_PI * dz) / dz)
    assert np.max(np.abs(q[11] - want)) <= 2e-14 * np.max(np.abs(want))


def test_gauss_law_outflow_linear_field():
    """E_x = x (and, in 2-D, E_y = 2 y): interior cells give the slope exactly;
    a boundary cell's outflow ghost equals the cell itself, so its central
    difference is half the slope."""
    nx = 10
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    E = np.stack([x[None, :], np.zeros((1, nx)), np.zeros((1, nx))])
    s = O.Sim(O.MODEL_SF, nx, 1, (0, 1), (0, 1), 2.0, 10.0, O.BC_OUTFLOW, O.BC_OUTFLOW)
    s.set_prims(_sf_prims_with_e(E, (1, nx)))
    rho = s.cons()[11, 0]
    want = np.ones(nx)
    want[0] = want[-1] = 0.5
    assert np.max(np.abs(rho - want)) <= 1e-14

    nx, ny = 9, 7
    dx, dy = 1.0 / nx, 1.0 / ny
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)
    E = np.stack([X, 2.0 * Y, np.zeros_like(X)])
    s = O.Sim(O.MODEL_SF, nx, ny, (0, 1), (0, 1), 2.0, 10.0, O.BC_OUTFLOW, O.BC_OUTFLOW)
    s.set_prims(_sf_prims_with_e(E, (ny, nx)))
    rho = s.cons()[11]
    wx = np.ones(nx)
    wx[0] = wx[-1] = 0.5
    wy = 2.0 * np.ones(ny)
    wy[0] = wy[-1] = 1.0
    assert np.max(np.abs(rho - (wx[None, :] + wy[:, None]))) <= 1e-13


def _expected_padded(interior, pads, modes):
    """np.pad of each variable's interior block, axis by axis (z, y, x)."""
    out = interior
    for ax, (p, m) in enumerate(zip(pads, modes)):
        if p == 0:
            continue
        width = [(0, 0)] * out.ndim
        width[ax + 1] = (p, p)
        out = np.pad(out, width, mode=m)
    return out


@pytest.mark.parametrize("bcs,shape", [
    ((O.BC_OUTFLOW, O.BC_OUTFLOW, None), (1, 9, 11)),
    ((O.BC_PERIODIC, O.BC_OUTFLOW, None), (1, 5, 7)),
    ((O.BC_OUTFLOW, O.BC_PERIODIC, None), (1, 6, 4)),
    ((O.BC_OUTFLOW, O.BC_OUTFLOW, None), (1, 1, 6)),      # 1-D: no y ghosts
    ((O.BC_PERIODIC, O.BC_PERIODIC, None), (1, 3, 1)),    # fewer cells than ghost layers
    ((O.BC_OUTFLOW, O.BC_PERIODIC, O.BC_OUTFLOW), (4, 5, 6)),
    ((O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_PERIODIC), (3, 4, 5)),
])
def test_ghost_cells_copy_or_wrap(bcs, shape):
    """Every ghost cell of the conserved state and of the primitives equals the
    nearest interior cell (outflow) or the periodic image (wrap), edges and
    corners included, after set_prims and again after a step."""
    bx, by, bz = bcs
    nz, ny, nx = shape
    rng = np.random.default_rng(7)
    n = nx * ny * nz
    P = np.zeros((11, n))
    P[0] = 1.0 + 0.2 * rng.random(n)
    P[1:4] = 0.1 * rng.uniform(-1, 1, (3, n))
    P[4] = 1.0 + 0.2 * rng.random(n)
    P[5:8] = 0.3 * rng.uniform(-1, 1, (3, n))
    P[8:11] = -np.cross(P[1:4].T, P[5:8].T).T  # E = -v x B
    kw = {}
    if nz > 1:
        kw = dict(nz=nz, zlim=(0, 1), bc_z=bz)
        P = P.reshape(11, nz, ny, nx)
    else:
        P = P.reshape(11, ny, nx)
    s = O.Sim(O.MODEL_SF, nx, ny, (0, 1), (0, 1), 4.0 / 3.0, 10.0, bx, by, **kw)
    s.set_prims(np.ascontiguousarray(P))
    mode = {O.BC_OUTFLOW: "edge", O.BC_PERIODIC: "wrap"}
    pads = (2 if nz > 1 else 0, 2 if ny > 1 else 0, 2)
    modes = (mode.get(bz, "edge"), mode[by], mode[bx])
    for rounds in range(2):
        for which, nv in (("cons", 14), ("prims", 5)):
            pad = s.padded(which)
            assert pad.shape == (nv, nz + 2 * pads[0], ny + 2 * pads[1], nx + 4)
            inner = pad[:, pads[0]:pads[0] + nz, pads[1]:pads[1] + ny, 2:2 + nx]
            assert np.array_equal(pad, _expected_padded(inner, pads, modes)), (which, rounds)
        s.step(1e-3, 1)
