"""FP64 PyTorch-CPU restatement of the SSP2(222) IMEX step of the resistive
single-fluid model, differentiable end to end with reverse-mode autograd: the
exact gradient of a functional of the final state with respect to the initial
primitives and the conductivity sigma, the oracle of the discrete adjoint.

TEST INFRASTRUCTURE: only tests/ import this module. It shares no code with the
CUDA library or with the C oracle (oracle/rmhd_oracle.c); it is written from
Wright & Hawke, arXiv:1808.09721, in plain tensor operations over all cells:

  - Eq. (resistive prims): primitives (rho, v, p, B, E) -> conserved
    (D, S, tau, B, E, varrho, psi, phi) with h = 1 + Gamma p / ((Gamma - 1) rho);
    at t = 0 varrho = div E (second-order central differences, ghosts by the
    boundary condition) and psi = phi = 0 (Sec. 2.1.1).
  - Sec. 2.1.3: primitive recovery. S~ = S - E x B, tau~ = tau - (E^2 + B^2)/2;
    the pressure solves f(p) = (Gamma - 1) rho eps - p = 0 with
    v = S~ / (tau~ + D + p), W = (1 - v^2)^(-1/2), rho = D / W,
    eps = (tau~ + D (1 - W) + p (1 - W^2)) / (D W).
  - Sec. 2.1.1: Ohm's law J = varrho v + W sigma [E + v x B - (v.E) v]; sources
    Psi_E = -J, Psi_psi = varrho - kappa psi, Psi_phi = -kappa phi, others 0;
    fluxes along k: D v^k; rho h W^2 v_i v^k + [p + (E^2 + B^2)/2] delta_ik
    - E_i E^k - B_i B^k; S^k - D v^k; B^i: -eps^{ijk} E_j + delta^k_i phi;
    E^i: eps^{ijk} B_j + delta^k_i psi; J^k; E^k; B^k.
  - Sec. 2.2.2: Lax-Friedrichs splitting f^+- = (f +- q)/2 (alpha = 1) and
    componentwise WENO3 in its textbook form (stencils p0, p1, smoothness
    beta0, beta1, linear weights 1/3, 2/3, epsilon = 1e-6, power 2);
    F = f^+_{i+1/2} + f^-_{i+1/2}, L_i = -sum_k (F_{i+1/2} - F_{i-1/2}) / dx_k.
  - Sec. 2.2.1, Eq. (implicit stage) and Table 1, SSP2(222) with
    gamma = 1 - 1/sqrt(2):
      q1 = q^n + gamma dt Psi(q1),
      q2 = q^n + dt L(q1) + dt [(1 - 2 gamma) Psi(q1) + gamma Psi(q2)],
      q^{n+1} = q^n + dt/2 [L(q1) + L(q2)] + dt/2 [Psi(q1) + Psi(q2)];
    and Table 2, SSP3(332) (ssp3_step: three implicit stages, weights 1/6,
    1/6, 2/3). Each implicit stage: components without a source equal r; psi, phi in
    closed form; E solves G(E) = E - r_E + a dt J(q(E)) = 0.
  - Boundary conditions: two ghost cells per side, outflow (copy the nearest
    interior cell) or periodic (wrap).

Roots. The pressure of every recovery and the E unknowns of every implicit
stage are found by Newton's method on detached values, iterated to a
round-off fixed point. One more Newton step is then taken with autograd on,
with the exact derivative of the residual in the unknown held constant. At a
converged root that step carries the derivative of the implicit-function
theorem, dx/dtheta = -(dG/dx)^-1 dG/dtheta (the term from differentiating the
step's slope is multiplied by the residual, which is zero), so the graph holds
the derivative of the discrete step without differentiating the iterations.
"""
from __future__ import annotations

import math

import torch

F64 = torch.float64
EPS_WENO = 1e-6
# conserved variable order of Eq. (resistive RMHD)
D, S0, TAU, B0, E0, RHOE, PSI, PHI, NC = 0, 1, 4, 5, 8, 11, 12, 13, 14
OUTFLOW, PERIODIC = 0, 1


def cross(a, b):
    return torch.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def dot(a, b):
    return (a * b).sum(0)


# ---- boundary conditions: ghost cells by index maps -----------------------
def _ghost_index(n, bc, g=2):
    i = torch.arange(-g, n + g)
    return i.remainder(n) if bc == PERIODIC else i.clamp(0, n - 1)


def pad(u, bcx, bcy, bcz=None):
    """u: (..., ny, nx) -> (..., ny + 4, nx + 4) (ny == 1: no ghosts along y);
    with bcz given, u: (..., nz, ny, nx) and ghosts along z too."""
    ny, nx = u.shape[-2], u.shape[-1]
    u = u.index_select(-1, _ghost_index(nx, bcx))
    if ny > 1:
        u = u.index_select(-2, _ghost_index(ny, bcy))
    if bcz is not None:
        u = u.index_select(-3, _ghost_index(u.shape[-3], bcz))
    return u


# ---- Eq. (resistive prims) -------------------------------------------------
def prims_to_cons(P, gamma, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    """P: (11, ny, nx), or (11, nz, ny, nx) for a 3-D grid."""
    rho, v, p, B, E = P[0], P[1:4], P[4], P[5:8], P[8:11]
    W = 1.0 / torch.sqrt(1.0 - dot(v, v))
    rhohW2 = (rho + gamma / (gamma - 1.0) * p) * W * W
    Dd = rho * W
    S = rhohW2 * v + cross(E, B)
    tau = rhohW2 - p + 0.5 * (dot(E, E) + dot(B, B)) - Dd
    # Gauss's law, second-order central differences
    if P.dim() == 4:  # 3-D
        Eg = pad(E, bcx, bcy, bcz)
        divE = ((Eg[0, 2:-2, 2:-2, 3:-1] - Eg[0, 2:-2, 2:-2, 1:-3]) / (2.0 * dx)
                + (Eg[1, 2:-2, 3:-1, 2:-2] - Eg[1, 2:-2, 1:-3, 2:-2]) / (2.0 * dy)
                + (Eg[2, 3:-1, 2:-2, 2:-2] - Eg[2, 1:-3, 2:-2, 2:-2]) / (2.0 * dz))
        z = torch.zeros_like(Dd)
        return torch.cat([Dd[None], S, tau[None], B, E, divE[None], z[None], z[None]])
    Eg = pad(E, bcx, bcy)
    ny = P.shape[1]
    divE = (Eg[0, :, 3:-1] - Eg[0, :, 1:-3]) / (2.0 * dx)
    if ny > 1:
        divE = divE[2:-2]
        divE = divE + (Eg[1, 3:-1, 2:-2] - Eg[1, 1:-3, 2:-2]) / (2.0 * dy)
    z = torch.zeros_like(Dd)
    return torch.cat([Dd[None], S, tau[None], B, E, divE[None], z[None], z[None]])


# ---- Sec. 2.1.3: primitive recovery ---------------------------------------
def _pressure_resid(p, Dd, St2, taut, gamma):
    Z = taut + Dd + p
    W = 1.0 / torch.sqrt(1.0 - St2 / (Z * Z))
    rho = Dd / W
    eps = (taut + Dd * (1.0 - W) + p * (1.0 - W * W)) / (Dd * W)
    return (gamma - 1.0) * rho * eps - p


def _pressure_root(Dd, St2, taut, gamma):
    """Newton with bisection safeguard on detached values, to a round-off fixed
    point. Returns the root and the slope df/dp there."""
    Dd, St2, taut = Dd.detach(), St2.detach(), taut.detach()
    lo = torch.clamp(torch.sqrt(St2) - taut - Dd, min=0.0)
    hi = torch.clamp((gamma - 1.0) * (taut + Dd), min=1e-300)
    with torch.no_grad():
        for _ in range(60):  # enlarge hi until f(hi) < 0 (f decreases through the root)
            bad = ~(_pressure_resid(hi, Dd, St2, taut, gamma) < 0)
            if not bool(bad.any()):
                break
            hi = torch.where(bad, 2.0 * hi, hi)
    p = 0.5 * (lo + hi)

    def f_and_slope(p):
        pr = p.clone().requires_grad_(True)
        with torch.enable_grad():
            f = _pressure_resid(pr, Dd, St2, taut, gamma)
            (df,) = torch.autograd.grad(f.sum(), pr)
        return f.detach(), df

    for _ in range(200):
        f, df = f_and_slope(p)
        lo = torch.where(f > 0, p, lo)
        hi = torch.where(f > 0, hi, p)
        pn = p - f / df
        pn = torch.where((pn > lo) & (pn < hi), pn, 0.5 * (lo + hi))
        done = (pn - p).abs() <= 4.0 * torch.finfo(F64).eps * p
        p = pn
        if bool(done.all()):
            break
    f, df = f_and_slope(p)
    if not bool(torch.isfinite(p).all()) or not bool((p > 0).all()):
        raise ArithmeticError("pressure root not found")
    return p, df


def recover(q, gamma):
    """Conserved -> (v, p, W); differentiable in q through the root's
    implicit-function derivative (one Newton step from the converged root)."""
    B, E, S = q[B0:B0 + 3], q[E0:E0 + 3], q[S0:S0 + 3]
    St = S - cross(E, B)
    taut = q[TAU] - 0.5 * (dot(E, E) + dot(B, B))
    St2 = dot(St, St)
    pd, slope = _pressure_root(q[D], St2, taut, gamma)
    p = pd - _pressure_resid(pd, q[D], St2, taut, gamma) / slope
    v = St / (taut + q[D] + p)
    W = 1.0 / torch.sqrt(1.0 - dot(v, v))
    return v, p, W


# ---- Sec. 2.1.1: Ohm's law, sources, fluxes --------------------------------
def current(q, v, W, sigma):
    E, B = q[E0:E0 + 3], q[B0:B0 + 3]
    return q[RHOE] * v + W * sigma * (E + cross(v, B) - dot(v, E) * v)


def source(q, v, W, sigma, kappa):
    s = torch.zeros_like(q)
    s = s.index_copy(0, torch.arange(E0, E0 + 3), -current(q, v, W, sigma))
    s = s.index_copy(0, torch.tensor([PSI, PHI]),
                     torch.stack([q[RHOE] - kappa * q[PSI], -kappa * q[PHI]]))
    return s


def flux(q, v, p, W, sigma, k):
    E, B = q[E0:E0 + 3], q[B0:B0 + 3]
    rhohW2 = q[TAU] - 0.5 * (dot(E, E) + dot(B, B)) + q[D] + p
    pem = p + 0.5 * (dot(E, E) + dot(B, B))
    J = current(q, v, W, sigma)
    rows = [q[D] * v[k]]
    for i in range(3):
        rows.append(rhohW2 * v[i] * v[k] + (pem if i == k else 0.0) - E[i] * E[k] - B[i] * B[k])
    rows.append(q[S0 + k] - q[D] * v[k])
    # B^i: -eps^{ijk} E_j + delta^k_i phi;  E^i: eps^{ijk} B_j + delta^k_i psi
    eps3 = {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}
    for i in range(3):
        val = q[PHI] if i == k else 0.0
        for j in range(3):
            val = val - eps3.get((i, j, k), 0) * E[j]
        rows.append(val if torch.is_tensor(val) else torch.zeros_like(q[D]))
    for i in range(3):
        val = q[PSI] if i == k else 0.0
        for j in range(3):
            val = val + eps3.get((i, j, k), 0) * B[j]
        rows.append(val if torch.is_tensor(val) else torch.zeros_like(q[D]))
    rows += [J[k], E[k], B[k]]
    return torch.stack(rows)


# ---- Sec. 2.2.2: LF splitting + WENO3 ---------------------------------------
def _weno3_plus(fm1, f0, fp1):
    """Face value f^+_{i+1/2} from f^+_{i-1}, f^+_i, f^+_{i+1}."""
    p0 = 0.5 * (-fm1 + 3.0 * f0)
    p1 = 0.5 * (f0 + fp1)
    b0 = (f0 - fm1) ** 2
    b1 = (fp1 - f0) ** 2
    a0 = (1.0 / 3.0) / (EPS_WENO + b0) ** 2
    a1 = (2.0 / 3.0) / (EPS_WENO + b1) ** 2
    return (a0 * p0 + a1 * p1) / (a0 + a1)


def _divergence_1d(qg, fg, h):
    """Along the last axis of padded arrays (n + 4 cells): -(F_{i+1/2} - F_{i-1/2}) / h
    for the n interior cells."""
    fp = 0.5 * (fg + qg)
    fmn = 0.5 * (fg - qg)
    n4 = qg.shape[-1]
    # faces i + 1/2 for padded i = 1 .. n + 1
    i = torch.arange(1, n4 - 2)
    Fp = _weno3_plus(fp[..., i - 1], fp[..., i], fp[..., i + 1])
    Fm = _weno3_plus(fmn[..., i + 2], fmn[..., i + 1], fmn[..., i])  # mirror image
    F = Fp + Fm
    return -(F[..., 1:] - F[..., :-1]) / h


def divergence(q, v, p, W, sigma, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    if q.dim() == 4:  # 3-D: (14, nz, ny, nx)
        qg, vg = pad(q, bcx, bcy, bcz), pad(v, bcx, bcy, bcz)
        pg, Wg = pad(p, bcx, bcy, bcz), pad(W, bcx, bcy, bcz)
        s_ = slice(2, -2)
        Lx = _divergence_1d(qg[:, s_, s_, :], flux(qg[:, s_, s_, :], vg[:, s_, s_, :], pg[s_, s_, :],
                                                   Wg[s_, s_, :], sigma, 0), dx)
        qy, fy = qg[:, s_, :, s_], flux(qg[:, s_, :, s_], vg[:, s_, :, s_], pg[s_, :, s_], Wg[s_, :, s_], sigma, 1)
        Ly = _divergence_1d(qy.transpose(2, 3), fy.transpose(2, 3), dy).transpose(2, 3)
        qz, fz = qg[:, :, s_, s_], flux(qg[:, :, s_, s_], vg[:, :, s_, s_], pg[:, s_, s_], Wg[:, s_, s_], sigma, 2)
        Lz = _divergence_1d(qz.permute(0, 2, 3, 1), fz.permute(0, 2, 3, 1), dz).permute(0, 3, 1, 2)
        return Lx + Ly + Lz
    ny = q.shape[1]
    qg = pad(q, bcx, bcy)
    vg, pg, Wg = pad(v, bcx, bcy), pad(p, bcx, bcy), pad(W, bcx, bcy)
    if ny == 1:
        return _divergence_1d(qg, flux(qg, vg, pg, Wg, sigma, 0), dx)
    Lx = _divergence_1d(qg[:, 2:-2], flux(qg[:, 2:-2], vg[:, 2:-2], pg[2:-2], Wg[2:-2], sigma, 0), dx)
    qt = qg[:, :, 2:-2].transpose(1, 2)
    ft = flux(qg[:, :, 2:-2], vg[:, :, 2:-2], pg[:, 2:-2], Wg[:, 2:-2], sigma, 1).transpose(1, 2)
    Ly = _divergence_1d(qt, ft, dy).transpose(1, 2)
    return Lx + Ly


# ---- Sec. 2.2.1: implicit stage --------------------------------------------
def _stage_q(r, E, adt, kappa):
    q = r.clone()
    q = q.index_copy(0, torch.arange(E0, E0 + 3), E)
    ck = 1.0 / (1.0 + adt * kappa)
    q = q.index_copy(0, torch.tensor([PSI, PHI]), torch.stack([(r[PSI] + adt * r[RHOE]) * ck, r[PHI] * ck]))
    return q


def _stage_G(r, E, adt, sigma, gamma, kappa):
    q = _stage_q(r, E, adt, kappa)
    v, p, W = recover(q, gamma)
    return E - r[E0:E0 + 3] + adt * current(q, v, W, sigma), q, (v, p, W)


def _scalar(x):
    return float(x.detach()) if torch.is_tensor(x) else float(x)


def _jacobian(r, E, adt, sigma, gamma, kappa):
    """dG/dE per cell, (..., 3, 3), by autograd on detached inputs."""
    Er = E.detach().clone().requires_grad_(True)
    with torch.enable_grad():
        G, _, _ = _stage_G(r.detach(), Er, adt, _scalar(sigma), gamma, kappa)
        rows = [torch.autograd.grad(G[i].sum(), Er, retain_graph=i < 2)[0] for i in range(3)]
    Jm = torch.stack(rows)  # [i][k][cells...] = dG_i/dE_k
    return G.detach(), Jm.movedim(0, -1).movedim(0, -1)  # (..., 3 (i), 3 (k))


def stage(r, adt, sigma, gamma, kappa):
    """q = r + adt Psi(q): Newton with backtracking on detached values to a
    round-off fixed point, then one differentiable Newton step."""
    rd = r.detach()
    E = rd[E0:E0 + 3].clone()
    scale = torch.maximum(torch.maximum(E.abs().amax(0), rd[B0:B0 + 3].abs().amax(0)), torch.full_like(E[0], 1e-300))
    for _ in range(60):
        G, Jm = _jacobian(rd, E, adt, sigma, gamma, kappa)
        dE = -torch.linalg.solve(Jm, G.movedim(0, -1).unsqueeze(-1)).squeeze(-1).movedim(-1, 0)
        m0 = (G * G).sum(0)
        t = torch.ones_like(m0)
        with torch.no_grad():
            for _ls in range(12):
                Gt, _, _ = _stage_G(rd, E + t * dE, adt, _scalar(sigma), gamma, kappa)
                ok = (Gt * Gt).sum(0) <= (1.0 - 1e-4 * t) * m0
                if bool(ok.all()):
                    break
                t = torch.where(ok, t, 0.5 * t)
        E = E + t * dE
        scale = torch.maximum(scale, E.abs().amax(0))
        if bool(((t * dE).abs().amax(0) <= 4.0 * torch.finfo(F64).eps * scale).all()):
            break
    G, Jm = _jacobian(rd, E, adt, sigma, gamma, kappa)
    Gd, q, _ = _stage_G(r, E, adt, sigma, gamma, kappa)  # differentiable in r and sigma
    step = torch.linalg.solve(Jm, Gd.movedim(0, -1).unsqueeze(-1)).squeeze(-1).movedim(-1, 0)
    Ef = E - step
    q = _stage_q(r, Ef, adt, kappa)
    v, p, W = recover(q, gamma)
    return q, (v, p, W)


# ---- Table 1: one SSP2(222) step ------------------------------------------
GAMMA_SSP2 = 1.0 - 1.0 / math.sqrt(2.0)


def ssp2_step(q, dt, sigma, gamma, kappa, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    g = GAMMA_SSP2
    q1, w1 = stage(q, g * dt, sigma, gamma, kappa)
    L1 = divergence(q1, *w1, sigma, bcx, bcy, dx, dy, bcz, dz)
    P1 = source(q1, w1[0], w1[2], sigma, kappa)
    r2 = q + dt * L1 + (1.0 - 2.0 * g) * dt * P1
    q2, w2 = stage(r2, g * dt, sigma, gamma, kappa)
    L2 = divergence(q2, *w2, sigma, bcx, bcy, dx, dy, bcz, dz)
    P2 = source(q2, w2[0], w2[2], sigma, kappa)
    return q + 0.5 * dt * (L1 + L2) + 0.5 * dt * (P1 + P2)


# ---- Table 2: one SSP3(332) step --------------------------------------------
def ssp3_step(q, dt, sigma, gamma, kappa, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    """Implicit rows (g, 0, 0), (1 - 2g, g, 0), (1/2 - g, 0, g); explicit rows
    (0, 0, 0), (1, 0, 0), (1/4, 1/4, 0); weights (1/6, 1/6, 2/3) for both parts."""
    g = GAMMA_SSP2
    q1, w1 = stage(q, g * dt, sigma, gamma, kappa)
    L1 = divergence(q1, *w1, sigma, bcx, bcy, dx, dy, bcz, dz)
    P1 = source(q1, w1[0], w1[2], sigma, kappa)
    q2, w2 = stage(q + dt * L1 + (1.0 - 2.0 * g) * dt * P1, g * dt, sigma, gamma, kappa)
    L2 = divergence(q2, *w2, sigma, bcx, bcy, dx, dy, bcz, dz)
    P2 = source(q2, w2[0], w2[2], sigma, kappa)
    q3, w3 = stage(q + 0.25 * dt * (L1 + L2) + (0.5 - g) * dt * P1, g * dt, sigma, gamma, kappa)
    L3 = divergence(q3, *w3, sigma, bcx, bcy, dx, dy, bcz, dz)
    P3 = source(q3, w3[0], w3[2], sigma, kappa)
    return q + dt / 6.0 * (L1 + P1) + dt / 6.0 * (L2 + P2) + 2.0 * dt / 3.0 * (L3 + P3)


def run(prims, sigma, dt, nsteps, gamma, bcx, bcy, dx, dy, kappa=1.0, scheme=0, bcz=1, dz=1.0):
    """prims (11, ny, nx), or (11, nz, ny, nx) for a 3-D grid, and sigma (0-d)
    as tensors (may require grad) -> q^n; scheme 0: SSP2(222), 1: SSP3(332)."""
    step = ssp3_step if scheme == 1 else ssp2_step
    q = prims_to_cons(prims, gamma, bcx, bcy, dx, dy, bcz, dz)
    for _ in range(nsteps):
        q = step(q, dt, sigma, gamma, kappa, bcx, bcy, dx, dy, bcz, dz)
    return q


def gradient(prims, sigma, dt, nsteps, gamma, bcx, bcy, dx, dy, lam, kappa=1.0, scheme=0, bcz=1, dz=1.0):
    """J = sum(lam * q^n): returns (J, dJ/dprims, dJ/dsigma) as NumPy/float."""
    P = torch.tensor(prims, dtype=F64, requires_grad=True)
    s = torch.tensor(float(sigma), dtype=F64, requires_grad=True)
    q = run(P, s, dt, nsteps, gamma, bcx, bcy, dx, dy, kappa, scheme, bcz, dz)
    J = (torch.tensor(lam, dtype=F64) * q).sum()
    gP, gs = torch.autograd.grad(J, (P, s))
    return float(J.detach()), gP.numpy(), float(gs), q.detach().numpy()


def jvp(prims, sigma, dt, nsteps, gamma, bcx, bcy, dx, dy, v_prims, v_sigma, kappa=1.0, scheme=0, bcz=1, dz=1.0):
    """Directional derivative of q^n along (v_prims, v_sigma): reverse mode
    applied twice. g(u) = d<u, q^n>/d(prims, sigma) is linear in u, so the
    derivative of <g(u), v> with respect to u is J v at any u."""
    P = torch.tensor(prims, dtype=F64, requires_grad=True)
    s = torch.tensor(float(sigma), dtype=F64, requires_grad=True)
    q = run(P, s, dt, nsteps, gamma, bcx, bcy, dx, dy, kappa, scheme, bcz, dz)
    u = torch.zeros_like(q, requires_grad=True)
    gP, gs = torch.autograd.grad((u * q).sum(), (P, s), create_graph=True)
    inner = (gP * torch.tensor(v_prims, dtype=F64)).sum() + gs * float(v_sigma)
    (Jv,) = torch.autograd.grad(inner, u)
    return Jv.numpy()
