"""Seeded synthetic initial data shaped like the paper's test problems.

This module only builds primitive fields (rho, v, p, B, E per species) and run
parameters; it holds none of the method's arithmetic (no conserved variables,
fluxes, sources or recovery). The CUDA library and the CPU oracle each turn
the same primitives into their own conserved state.

Workloads (paper sections in brackets):
  brio_wu      1-D shock tube, one fluid, N = 400, sigma = 100, Gamma = 2   [Sec. 4.1]
  khi          2-D Kelvin-Helmholtz shear layer, 1024^2 periodic, sigma = 1e3 [Sec. 4.4]
  tf_sheet     2-D two-fluid pair-plasma current sheet, 512^2 periodic        [Sec. 4.2-4.3]
  batch_tubes  512 independent 1-D shock tubes of uneven size and sigma        [Sec. 4.1]
  field_loop   2-D field-loop advection, 256^2 periodic                        [Sec. 4.3]
  current_sheet 1-D self-similar resistive current sheet                      [Sec. 4.2]
Electric fields are set to the ideal-MHD value E = -v x B of the local bulk
velocity, so the initial state carries no artificial resistive current.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

RESISTIVE, TWO_FLUID = 0, 1
OUTFLOW, PERIODIC = 0, 1


@dataclass
class Workload:
    name: str
    model: int
    nx: int
    ny: int
    xlim: tuple
    ylim: tuple
    gamma: float
    sigma: float
    bc_x: int
    bc_y: int
    cfl: float
    nsteps: int
    prims: np.ndarray = field(repr=False)  # [n_prim][ny][nx] ([n_prim][nz][ny][nx] in 3-D) float64
    mu_e: float = -1.0
    mu_p: float = 1.0
    kappa: float = 1.0
    nz: int = 1
    zlim: tuple = (0.0, 1.0)
    bc_z: int = 1

    @property
    def dx(self):
        return (self.xlim[1] - self.xlim[0]) / self.nx

    @property
    def dy(self):
        return (self.ylim[1] - self.ylim[0]) / self.ny

    @property
    def dz(self):
        return (self.zlim[1] - self.zlim[0]) / self.nz

    @property
    def dt(self):
        h = self.dx if self.ny == 1 else min(self.dx, self.dy)
        if self.nz > 1:
            h = min(h, self.dz)
        return self.cfl * h

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def with_prims(self, prims, **kw):
        return replace(self, prims=prims, **kw)


def _centres(lo, hi, n):
    return lo + (np.arange(n) + 0.5) * (hi - lo) / n


def _ideal_e(v, B):
    """E = -v x B, componentwise over fields of shape (3, ...)."""
    return -np.stack([v[1] * B[2] - v[2] * B[1],
                      v[2] * B[0] - v[0] * B[2],
                      v[0] * B[1] - v[1] * B[0]])


def _sf_prims(rho, v, p, B, E):
    return np.ascontiguousarray(np.concatenate([rho[None], v, p[None], B, E]).astype(np.float64))


def brio_wu(nx: int = 400, sigma: float = 100.0, gamma: float = 2.0, bx: float = 0.5,
            by: float = 1.0, cfl: float = 0.4) -> Workload:
    """Shock tube on x in [0, 1]: left (rho, p, B_y) = (1, 1, by), right (0.125, 0.1, -by),
    B_x = bx, v = 0, E = 0; outflow; 400 steps of dt = cfl/nx reach t = 0.4 at N = 400."""
    x = _centres(0.0, 1.0, nx)[None, :]
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(x)
    B = np.stack([z + bx, np.where(left, by, -by), z])
    v = np.stack([z, z, z])
    E = _ideal_e(v, B)
    nsteps = int(round(0.4 / (cfl / nx)))
    return Workload("brio_wu", RESISTIVE, nx, 1, (0.0, 1.0), (0.0, 1.0), gamma, sigma,
                    OUTFLOW, OUTFLOW, cfl, nsteps, _sf_prims(rho, v, p, B, E))


def khi(n: int = 1024, seed: int = 0, sigma: float = 1e3, gamma: float = 4.0 / 3.0,
        a: float = 0.01, cfl: float = 0.4, nsteps: int = 200, ny: int | None = None) -> Workload:
    """Kelvin-Helmholtz shear layer on [-1/2, 1/2]^2, periodic:
    rho = 1 - 0.9 * band, band = [tanh((y+1/4)/a) - tanh((y-1/4)/a)]/2 (rho = 0.1 for |y| < 1/4),
    v_x = 0.25 (2 band - 1), v_y = 1e-3 U(-1, 1) (seeded), p = 1, B = (0.1, 0, 0)."""
    ny = n if ny is None else ny
    x = _centres(-0.5, 0.5, n)
    y = _centres(-0.5, 0.5, ny)
    Y, X = np.meshgrid(y, x, indexing="ij")
    band = 0.5 * (np.tanh((Y + 0.25) / a) - np.tanh((Y - 0.25) / a))
    rho = 1.0 - 0.9 * band
    rng = np.random.default_rng(seed)
    vx = 0.25 * (2.0 * band - 1.0)
    vy = 1e-3 * rng.uniform(-1.0, 1.0, size=X.shape)
    z = np.zeros_like(X)
    v = np.stack([vx, vy, z])
    p = np.ones_like(X)
    B = np.stack([z + 0.1, z, z])
    E = _ideal_e(v, B)
    return Workload("khi", RESISTIVE, n, ny, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, nsteps, _sf_prims(rho, v, p, B, E))


def khi3d(n: int = 128, seed: int = 0, sigma: float = 1e3, gamma: float = 4.0 / 3.0,
          a: float = 0.05, cfl: float = 0.4, nsteps: int = 50, shape=None) -> Workload:
    """3-D Kelvin-Helmholtz shear layer on [-1/2, 1/2]^3, periodic: the KHI
    recipe of `khi` extended along z (rho and v_x depend on y), seeded noise
    1e-3 U(-1, 1) on v_y and v_z, p = 1, B = (0.1, 0, 0), E = -v x B.
    `shape` = (nz, ny, nx) for a non-cubic grid."""
    nz, ny, nx = (n, n, n) if shape is None else shape
    x = _centres(-0.5, 0.5, nx)
    y = _centres(-0.5, 0.5, ny)
    zc = _centres(-0.5, 0.5, nz)
    Z, Y, X = np.meshgrid(zc, y, x, indexing="ij")
    band = 0.5 * (np.tanh((Y + 0.25) / a) - np.tanh((Y - 0.25) / a))
    rng = np.random.default_rng(seed)
    rho = 1.0 - 0.9 * band
    v = np.stack([0.25 * (2.0 * band - 1.0), 1e-3 * rng.uniform(-1.0, 1.0, size=X.shape),
                  1e-3 * rng.uniform(-1.0, 1.0, size=X.shape)])
    zero = np.zeros_like(X)
    B = np.stack([zero + 0.1, zero, zero])
    prims = _sf_prims(rho, v, np.ones_like(X), B, _ideal_e(v, B))
    return Workload("khi3d", RESISTIVE, nx, ny, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, nsteps, prims, nz=nz, zlim=(-0.5, 0.5), bc_z=PERIODIC)


def tf_sheet(n: int = 512, seed: int = 1, sigma: float = 1e4, mu: float = 1e3,
             gamma: float = 4.0 / 3.0, width: float = 0.05, cfl: float = 0.4,
             nsteps: int = 100, ny: int | None = None) -> Workload:
    """Two-fluid pair-plasma current sheet on [-1/2, 1/2]^2, periodic: per species
    rho_s = 1/2, p_s = 1/2 (totals 1, 1), v_y,s = 1e-4 U(-1, 1) (independent draws),
    B_y = tanh(x / width), mu_e = -mu, mu_p = +mu; E = -vbar x B with vbar the
    mean species velocity. The periodic wrap forms a second sheet at x = +-1/2."""
    ny = n if ny is None else ny
    x = _centres(-0.5, 0.5, n)
    y = _centres(-0.5, 0.5, ny)
    Y, X = np.meshgrid(y, x, indexing="ij")
    rng = np.random.default_rng(seed)
    z = np.zeros_like(X)
    half = np.full_like(X, 0.5)
    ve = np.stack([z, 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape), z])
    vp = np.stack([z, 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape), z])
    B = np.stack([z, np.tanh(X / width), z])
    E = _ideal_e(0.5 * (ve + vp), B)
    prims = np.concatenate([half[None], ve, half[None], half[None], vp, half[None], B, E]).astype(np.float64)
    return Workload("tf_sheet", TWO_FLUID, n, ny, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, nsteps, np.ascontiguousarray(prims), mu_e=-mu, mu_p=mu)


def _tf_species_prims(rho, p, v, B, E, mu_e, mu_p):
    """Neutral two-species plasma from totals: equal number densities (charges
    +-q, so masses m_s ~ 1/|mu_s| and rho_p / rho_e = |mu_e / mu_p|), equal
    temperatures (p_s = p / 2), both species moving with v."""
    frac_e = abs(mu_p) / (abs(mu_e) + abs(mu_p))
    return np.concatenate([(frac_e * rho)[None], v, (0.5 * p)[None],
                           ((1.0 - frac_e) * rho)[None], v, (0.5 * p)[None], B, E]).astype(np.float64)


def _smooth(rng, coords, amp, nmodes=3):
    """Sum of nmodes random periodic Fourier modes (integer wave numbers 1..2
    per axis on the unit-length axes `coords`), scaled to max |f| = amp."""
    f = np.zeros(coords[0].shape)
    for _ in range(nmodes):
        k = rng.integers(0, 3, size=len(coords))
        k[rng.integers(0, len(coords))] = rng.integers(1, 3)  # at least one nonzero wave number
        phase = rng.uniform(0.0, 2.0 * np.pi)
        f = f + rng.uniform(0.5, 1.0) * np.sin(2.0 * np.pi * sum(ki * c for ki, c in zip(k, coords)) + phase)
    return amp * f / max(np.max(np.abs(f)), 1e-300)


def random_smooth(shape, seed: int = 0, model: int = RESISTIVE, sigma: float = 10.0,
                  gamma: float = 4.0 / 3.0, cfl: float = 0.4, bc: int = PERIODIC,
                  mu: float = 1e3) -> Workload:
    """Smooth random periodic fields on the unit box with every component
    nonzero: rho, p in [0.5, 1.5], |v_i| <= 0.3, |B_i| <= 1 and
    E = -v x B + dE with a smooth |dE_i| <= 0.1 (a resistive current). `shape`
    = (nx,), (ny, nx) or (nz, ny, nx). Two fluids: the totals split into a
    neutral pair plasma (mu_p = -mu_e = mu), the positive species' velocity
    offset by a smooth |dv_i| <= 0.05 (a current carried by the species)."""
    shape = tuple(shape)
    nd = len(shape)
    nz, ny, nx = (1,) * (3 - nd) + shape
    axes = [(np.arange(n) + 0.5) / n for n in (nz, ny, nx)]
    Z, Y, X = np.meshgrid(*axes, indexing="ij")
    coords = [X, Y, Z][:nd]
    rng = np.random.default_rng(seed)
    rho = 1.0 + _smooth(rng, coords, 0.5)
    p = 1.0 + _smooth(rng, coords, 0.5)
    v = np.stack([_smooth(rng, coords, 0.3) for _ in range(3)])
    B = np.stack([_smooth(rng, coords, 1.0) for _ in range(3)])
    E = _ideal_e(v, B) + np.stack([_smooth(rng, coords, 0.1) for _ in range(3)])
    sq = (lambda a: a.reshape(a.shape[:-3] + (ny, nx))) if nz == 1 else (lambda a: a)
    kw = dict(nz=nz, zlim=(0.0, 1.0), bc_z=bc) if nz > 1 else {}
    if model == RESISTIVE:
        prims = _sf_prims(sq(rho), sq(v), sq(p), sq(B), sq(E))
        return Workload("random_smooth", RESISTIVE, nx, ny, (0.0, 1.0), (0.0, 1.0), gamma, sigma, bc, bc,
                        cfl, 10, prims, **kw)
    sp = _tf_species_prims(sq(rho), sq(p), sq(v), sq(B), sq(E), -mu, mu)
    dv = np.stack([_smooth(rng, coords, 0.05) for _ in range(3)])
    sp[6:9] += sq(dv)  # positive species' velocity (rows: rho_e, v_e, p_e, rho_p, v_p, p_p, B, E)
    return Workload("random_smooth_tf", TWO_FLUID, nx, ny, (0.0, 1.0), (0.0, 1.0), gamma, sigma, bc, bc,
                    cfl, 10, np.ascontiguousarray(sp), mu_e=-mu, mu_p=mu, **kw)


def relativistic_smooth(shape, seed: int = 0, sigma: float = 1e8, wmax: float = 10.0, gamma: float = 4.0 / 3.0,
                        cfl: float = 0.4, bc: int = PERIODIC) -> Workload:
    """Smooth random periodic single-fluid fields in relativistic bulk motion:
    rho, p in [0.5, 1.5], B_i up to 1, a velocity of one random direction
    (perturbed by up to 5% per component) with Lorentz factor W varying
    smoothly by 10% around wmax (|v| = sqrt(1 - 1/W^2)), and E = -v x B + a
    smooth |dE_i| <= 0.1 (a resistive current that stiff sigma damps)."""
    shape = tuple(shape)
    nd = len(shape)
    nz, ny, nx = (1,) * (3 - nd) + shape
    axes = [(np.arange(n) + 0.5) / n for n in (nz, ny, nx)]
    Z, Y, X = np.meshgrid(*axes, indexing="ij")
    coords = [X, Y, Z][:nd]
    rng = np.random.default_rng(seed)
    rho = 1.0 + _smooth(rng, coords, 0.5)
    p = 1.0 + _smooth(rng, coords, 0.5)
    d0 = rng.standard_normal(3)
    d = np.stack([d0[i] / np.linalg.norm(d0) + _smooth(rng, coords, 0.05) for i in range(3)])
    d = d / np.sqrt((d * d).sum(axis=0))
    W = wmax * (1.0 + _smooth(rng, coords, 0.1))
    v = d * np.sqrt(1.0 - 1.0 / (W * W))
    B = np.stack([_smooth(rng, coords, 1.0) for _ in range(3)])
    E = _ideal_e(v, B) + np.stack([_smooth(rng, coords, 0.1) for _ in range(3)])
    sq = (lambda a: a.reshape(a.shape[:-3] + (ny, nx))) if nz == 1 else (lambda a: a)
    kw = dict(nz=nz, zlim=(0.0, 1.0), bc_z=bc) if nz > 1 else {}
    prims = _sf_prims(sq(rho), sq(v), sq(p), sq(B), sq(E))
    return Workload("relativistic_smooth", RESISTIVE, nx, ny, (0.0, 1.0), (0.0, 1.0), gamma, sigma, bc, bc,
                    cfl, 10, prims, **kw)


def tf_brio_wu(nx: int = 1600, mu_p: float = 1e3, mass_ratio: float = 1.0, sigma: float = 1e4,
               gamma: float = 2.0, cfl: float = 0.4) -> Workload:
    """Two-fluid Brio-Wu tube (Sec. 4.1): x in [0, 1], outflow, (rho, p, B_x, B_y) =
    (1, 1, 0.5, 1) left and (0.125, 0.1, 0.5, -1) right of x = 1/2, v = 0, E = 0,
    run to T = 0.4. mu_p = 1e3; mu_e = -mass_ratio * mu_p (1: pair plasma; 100:
    electron-proton). sigma (eta = 1/sigma) and Gamma are not printed: 1e4 and 2."""
    x = _centres(0.0, 1.0, nx)[None, :]
    left = x < 0.5
    z = np.zeros_like(x)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    B = np.stack([z + 0.5, np.where(left, 1.0, -1.0), z])
    v = np.stack([z, z, z])
    mu_e = -mass_ratio * mu_p
    prims = _tf_species_prims(rho, p, v, B, np.stack([z, z, z]), mu_e, mu_p)
    dt = cfl / nx
    return Workload("tf_brio_wu", TWO_FLUID, nx, 1, (0.0, 1.0), (0.0, 1.0), gamma, sigma,
                    OUTFLOW, OUTFLOW, cfl, int(round(0.4 / dt)), np.ascontiguousarray(prims),
                    mu_e=mu_e, mu_p=mu_p)


def tf_current_sheet(nx: int = 50, mu: float = 1e3, sigma: float = 100.0, t0: float = 1.0, b0: float = 1.0,
                     xlim=(-1.5, 1.5), gamma: float = 2.0, cfl: float = 0.4, p: float = 50.0) -> Workload:
    """Two-fluid self-similar current sheet (Sec. 4.2), pair plasma mu = +-1e3:
    rho = 1, p = 50 (halves per species), v = 0, E = 0, B_y = b0 erf(x sqrt(sigma / t0) / 2)."""
    x = _centres(xlim[0], xlim[1], nx)[None, :]
    z = np.zeros_like(x)
    by = b0 * np.vectorize(math.erf)(0.5 * x * math.sqrt(sigma / t0))
    prims = _tf_species_prims(np.ones_like(x), np.full_like(x, p), np.stack([z, z, z]), np.stack([z, by, z]),
                              np.stack([z, z, z]), -mu, mu)
    return Workload("tf_current_sheet", TWO_FLUID, nx, 1, xlim, (0.0, 1.0), gamma, sigma,
                    OUTFLOW, OUTFLOW, cfl, 0, np.ascontiguousarray(prims), mu_e=-mu, mu_p=mu)


def tf_sheet3d(shape=(64, 64, 64), seed: int = 1, sigma: float = 1e4, mu: float = 1e3,
               gamma: float = 4.0 / 3.0, width: float = 0.05, cfl: float = 0.4, nsteps: int = 20) -> Workload:
    """The two-fluid pair-plasma current sheet of `tf_sheet` on [-1/2, 1/2]^3,
    periodic, (nz, ny, nx) = shape: B_y = tanh(x / width), per species
    rho_s = p_s = 1/2, seeded 1e-4 U(-1, 1) noise on v_y and v_z of each species."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(_centres(-0.5, 0.5, nz), _centres(-0.5, 0.5, ny), _centres(-0.5, 0.5, nx),
                          indexing="ij")
    rng = np.random.default_rng(seed)
    z = np.zeros_like(X)
    half = np.full_like(X, 0.5)
    ve = np.stack([z, 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape), 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape)])
    vp = np.stack([z, 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape), 1e-4 * rng.uniform(-1.0, 1.0, size=X.shape)])
    B = np.stack([z, np.tanh(X / width), z])
    E = _ideal_e(0.5 * (ve + vp), B)
    prims = np.concatenate([half[None], ve, half[None], half[None], vp, half[None], B, E]).astype(np.float64)
    return Workload("tf_sheet3d", TWO_FLUID, nx, ny, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, nsteps, np.ascontiguousarray(prims), mu_e=-mu, mu_p=mu,
                    nz=nz, zlim=(-0.5, 0.5), bc_z=PERIODIC)


def batch_tubes(count: int = 512, seed: int = 2, nmin: int = 100, nmax: int = 4096,
                gamma: float = 4.0 / 3.0, cfl: float = 0.4, nsteps: int = 400) -> list:
    """Independent 1-D shock tubes on [0, 1], outflow: N ~ U{nmin..nmax},
    sigma log-uniform in [1, 1e6], rho_L, rho_R, p_L, p_R log-uniform in [0.1, 10],
    B_y = +1 left / -1 right, B_x = 0.5, v = 0. Each tube keeps its own dt = cfl / N."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        sigma = float(10.0 ** rng.uniform(0.0, 6.0))
        rl, rr, pl, pr = (float(10.0 ** rng.uniform(-1.0, 1.0)) for _ in range(4))
        x = _centres(0.0, 1.0, n)[None, :]
        left = x < 0.5
        z = np.zeros_like(x)
        rho = np.where(left, rl, rr)
        p = np.where(left, pl, pr)
        B = np.stack([z + 0.5, np.where(left, 1.0, -1.0), z])
        v = np.stack([z, z, z])
        out.append(Workload(f"tube{b}", RESISTIVE, n, 1, (0.0, 1.0), (0.0, 1.0), gamma, sigma,
                            OUTFLOW, OUTFLOW, cfl, nsteps, _sf_prims(rho, v, p, B, _ideal_e(v, B))))
    return out


def field_loop(n: int = 256, seed: int = 3, gamma: float = 2.0, cfl: float = 0.4,
               nsteps: int = 50, amp: float = 1e-3, radius: float = 0.3,
               v=(0.5, 0.25, 0.0)) -> Workload:
    """Field-loop advection on [-1/2, 1/2]^2, periodic: A_z = amp (radius - r) for r < radius,
    sampled at cell corners; B = curl(A_z z) with corner differences averaged to cell
    centres (discrete div B = 0 up to round-off); rho = p = 1, uniform v;
    sigma = 10^U(1, 4) drawn from the seed."""
    rng = np.random.default_rng(seed)
    sigma = float(10.0 ** rng.uniform(1.0, 4.0))
    h = 1.0 / n
    xc = -0.5 + np.arange(n + 1) * h  # corners
    Yc, Xc = np.meshgrid(xc, xc, indexing="ij")
    r = np.sqrt(Xc ** 2 + Yc ** 2)
    A = np.where(r < radius, amp * (radius - r), 0.0)
    # B_x = dA/dy, B_y = -dA/dx at centres (average of the two corner differences)
    bx = 0.5 * ((A[1:, :-1] - A[:-1, :-1]) + (A[1:, 1:] - A[:-1, 1:])) / h
    by = -0.5 * ((A[:-1, 1:] - A[:-1, :-1]) + (A[1:, 1:] - A[1:, :-1])) / h
    z = np.zeros((n, n))
    B = np.stack([bx, by, z])
    vv = np.stack([z + v[0], z + v[1], z + v[2]])
    prims = _sf_prims(np.ones((n, n)), vv, np.ones((n, n)), B, _ideal_e(vv, B))
    return Workload("field_loop", RESISTIVE, n, n, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, nsteps, prims)


def field_loop_bz(n: int = 64, b0: float = 1e-3, radius: float = 0.3, sigma: float = 1e5,
                  gamma: float = 2.0, cfl: float = 0.4, rho: float = 3.0, p: float = 1.0,
                  v=(0.1, 0.1, 0.0), shift: float = 0.0) -> Workload:
    """Field loop of the convergence test (Sec. 4.3): on [-1/2, 1/2]^2, periodic,
    rho = 3, v = (0.1, 0.1, 0), p = 1, B_z = b0 (R - r) for r <= R, else 0 (b0 = 1e-3;
    R is not printed: 0.3), E = -v x B, sigma = 1e5, Gamma = 2. `shift` = t samples
    the exactly advected profile B_z(x - v t) instead (uniform v: pure advection)."""
    h = 1.0 / n
    xc = -0.5 + (np.arange(n) + 0.5) * h
    Y, X = np.meshgrid(xc, xc, indexing="ij")
    X = (X - v[0] * shift + 0.5) % 1.0 - 0.5
    Y = (Y - v[1] * shift + 0.5) % 1.0 - 0.5
    r = np.sqrt(X ** 2 + Y ** 2)
    z = np.zeros((n, n))
    B = np.stack([z, z, np.where(r <= radius, b0 * (radius - r), 0.0)])
    vv = np.stack([z + v[0], z + v[1], z + v[2]])
    prims = _sf_prims(np.full((n, n), rho), vv, np.full((n, n), p), B, _ideal_e(vv, B))
    return Workload("field_loop_bz", RESISTIVE, n, n, (-0.5, 0.5), (-0.5, 0.5), gamma, sigma,
                    PERIODIC, PERIODIC, cfl, 0, prims)


def current_sheet(nx: int = 100, sigma: float = 100.0, t0: float = 1.0, b0: float = 1.0,
                  xlim=(-1.5, 1.5), gamma: float = 2.0, cfl: float = 0.4,
                  p: float = 50.0) -> Workload:
    """Self-similar current sheet (one fluid): rho = 1, p = 50, v = 0, E = 0,
    B_y = b0 erf(x sqrt(sigma / t0) / 2) -- the diffusion profile with eta = 1/sigma at t0."""
    x = _centres(xlim[0], xlim[1], nx)[None, :]
    z = np.zeros_like(x)
    by = b0 * np.vectorize(math.erf)(0.5 * x * math.sqrt(sigma / t0))
    B = np.stack([z, by, z])
    v = np.stack([z, z, z])
    prims = _sf_prims(np.ones_like(x), v, np.full_like(x, p), B, np.stack([z, z, z]))
    return Workload("current_sheet", RESISTIVE, nx, 1, xlim, (0.0, 1.0), gamma, sigma,
                    OUTFLOW, OUTFLOW, cfl, 0, prims)


def random_sf_states(n: int, seed: int, wmax: float = 10.0, theta=(1e-2, 1e2), emax: float = 1.0,
                     bmax: float = 1.0):
    """Random admissible single-fluid primitive cells (n, 11): Lorentz factor in
    [1, wmax], p/rho log-uniform in theta, |E| <= emax, |B| <= bmax."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 11))
    for k in range(n):
        W = 1.0 + (wmax - 1.0) * rng.uniform() ** 2
        speed = math.sqrt(1.0 - 1.0 / W ** 2)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        rho = 10.0 ** rng.uniform(-1.0, 1.0)
        p = rho * 10.0 ** rng.uniform(math.log10(theta[0]), math.log10(theta[1]))
        B = rng.normal(size=3)
        B *= bmax * rng.uniform() / np.linalg.norm(B)
        E = rng.normal(size=3)
        E *= emax * rng.uniform() / np.linalg.norm(E)
        out[k] = [rho, *(speed * d), p, *B, *E]
    return out


def random_tf_states(n: int, seed: int, wmax: float = 5.0, emax: float = 1.0, bmax: float = 1.0,
                     drift: float | None = None):
    """Random admissible two-fluid primitive cells (n, 16). With drift=None the
    species are independent; otherwise both species share a bulk velocity and
    differ by at most `drift` per component, densities agree to 1e-3 (a nearly
    neutral pair plasma), temperatures p/rho lie in [0.3, 30] and agree within a
    factor 2, and E is the ideal field -vbar x B of
    the mean velocity plus a perturbation of size 0.2 * drift * emax."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 16))
    for k in range(n):
        row = []
        W = 1.0 + (wmax - 1.0) * rng.uniform() ** 2
        bulk = math.sqrt(1.0 - 1.0 / W ** 2) * rng.normal(size=3)
        bulk *= math.sqrt(1.0 - 1.0 / W ** 2) / np.linalg.norm(bulk)
        rho0 = 10.0 ** rng.uniform(-1.0, 0.5)
        theta0 = 10.0 ** rng.uniform(-0.5, 1.5)
        for _ in range(2):
            if drift is None:
                W = 1.0 + (wmax - 1.0) * rng.uniform() ** 2
                speed = math.sqrt(1.0 - 1.0 / W ** 2)
                d = rng.normal(size=3)
                v = speed * d / np.linalg.norm(d)
                rho = 10.0 ** rng.uniform(-1.0, 0.5)
            else:
                v = bulk * 0.95 + drift * rng.uniform(-1.0, 1.0, size=3)
                rho = rho0 * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0))
            if drift is None:
                p = rho * 10.0 ** rng.uniform(-1.5, 1.5)
            else:
                p = rho * theta0 * 2.0 ** rng.uniform(-0.5, 0.5)
            row += [rho, *v, p]
        B = rng.normal(size=3)
        B *= bmax * rng.uniform() / np.linalg.norm(B)
        E = rng.normal(size=3)
        E *= emax * rng.uniform() / np.linalg.norm(E)
        if drift is not None:
            vbar = 0.5 * (np.array(row[1:4]) + np.array(row[6:9]))
            E = -np.cross(vbar, B) + drift * 0.2 * E
        out[k] = row + [*B, *E]
    return out
