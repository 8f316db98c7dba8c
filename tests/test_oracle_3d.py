"""Pins of the oracle's 3-D grids (nz > 1; the flux divergence of Sec. 2.2.2
summed over x, y and z): a tube along z equals the rotated tube along x,
periodic totals are conserved, and a constant state has zero divergence."""
import numpy as np

import oracle as O
from paper_1808_09721_gb300 import workloads as WL


def _cyc2(v):
    """Components of a vector in axes where the old x axis becomes z:
    (V_x, V_y, V_z) -> (V_y, V_z, V_x), an orientation-preserving rotation."""
    return np.stack([v[1], v[2], v[0]])


def _rot_prims(p):
    return np.concatenate([p[0:1], _cyc2(p[1:4]), p[4:5], _cyc2(p[5:8]), _cyc2(p[8:11])])


def _rot_cons(q):
    return np.concatenate([q[0:1], _cyc2(q[1:4]), q[4:5], _cyc2(q[5:8]), _cyc2(q[8:11]), q[11:14]])


def test_tube_along_z_equals_tube_along_x():
    n, m = 40, 4
    wl = WL.brio_wu(nx=n)
    p = wl.prims[:, 0, :]                                    # (11, n) along x
    sx = O.Sim(O.MODEL_SF, n, m, (0, 1), (0, 0.1), wl.gamma, wl.sigma, O.BC_OUTFLOW, O.BC_PERIODIC,
               nz=m, zlim=(0, 0.1), bc_z=O.BC_PERIODIC)
    sx.set_prims(np.ascontiguousarray(np.broadcast_to(p[:, None, None, :], (11, m, m, n))))
    pz = _rot_prims(p)
    sz = O.Sim(O.MODEL_SF, m, m, (0, 0.1), (0, 0.1), wl.gamma, wl.sigma, O.BC_PERIODIC, O.BC_PERIODIC,
               nz=n, zlim=(0, 1), bc_z=O.BC_OUTFLOW)
    sz.set_prims(np.ascontiguousarray(np.broadcast_to(pz[:, :, None, None], (11, n, m, m))))
    dt = 0.4 * (1.0 / n) * 0.25
    sx.step(dt, 5)
    sz.step(dt, 5)
    qx = sx.cons()[:, 0, 0, :]
    qz = sz.cons()[:, :, 0, 0]
    want = _rot_cons(qx)
    scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-12)
    assert np.max(np.abs(want - qz) / scale) <= 1e-13
    # the transverse directions stay uniform
    assert np.max(np.abs(sz.cons() - qz[:, :, None, None])) <= 1e-14 * np.abs(qz).max()


def test_conservation_periodic_3d():
    rng = np.random.default_rng(7)
    nx, ny, nz = 8, 6, 5
    z = np.zeros((nz, ny, nx))
    v = 0.2 * rng.uniform(-1, 1, size=(3, nz, ny, nx))
    B = rng.uniform(-1, 1, size=(3, nz, ny, nx))
    E = -np.stack([v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]])
    prims = np.concatenate([(1.0 + 0.1 * rng.uniform(size=(nz, ny, nx)))[None], v, (1.0 + z)[None], B, E])
    s = O.Sim(O.MODEL_SF, nx, ny, (0, 1), (0, 0.75), 4.0 / 3.0, 1e3, O.BC_PERIODIC, O.BC_PERIODIC,
              nz=nz, zlim=(0, 0.625), bc_z=O.BC_PERIODIC)
    s.set_prims(np.ascontiguousarray(prims))
    c0 = s.cons()
    a0 = np.abs(c0).reshape(14, -1).sum(axis=1)
    s0 = c0.reshape(14, -1).sum(axis=1)
    s.step(0.4 * 0.125 * 0.5, 3)
    s1 = s.cons().reshape(14, -1).sum(axis=1)
    for k in (0, 1, 2, 3, 4, 5, 6, 7, 11):
        assert abs(s1[k] - s0[k]) <= 1e-13 * max(a0[k], 1.0), (k, s1[k] - s0[k])


def test_constant_state_has_zero_divergence_3d():
    prim = np.array([1.0, 0.3, -0.2, 0.1, 2.0, 0.4, 0.2, -0.5, 0.0, 0.0, 0.0])
    v, B = prim[1:4], prim[5:8]
    prim[8:11] = -np.cross(v, B)
    s = O.Sim(O.MODEL_SF, 5, 4, (0, 1), (0, 1), 4.0 / 3.0, 10.0, O.BC_PERIODIC, O.BC_OUTFLOW,
              nz=6, bc_z=O.BC_PERIODIC)
    s.set_prims(np.ascontiguousarray(np.broadcast_to(prim[:, None, None, None], (11, 6, 4, 5))))
    assert np.max(np.abs(s.flux_divergence())) == 0.0
