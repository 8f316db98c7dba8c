"""FP64 PyTorch-CPU restatement of the SSP2(222) and SSP3(332) IMEX steps of
the two-fluid model, differentiable end to end with reverse-mode autograd: the
exact gradient of a functional of the final state with respect to the initial
primitives and the conductivity sigma, the oracle of the two-fluid discrete
adjoint.

TEST INFRASTRUCTURE: only tests/ import this module. It shares no code with the
CUDA library or with the C oracle (oracle/rmhd_oracle.c); it is written from
Wright & Hawke, arXiv:1808.09721, in plain tensor operations over all cells,
and takes from oracle/autodiff_sf.py only what the two models have in common
(ghost cells, the LF/WENO3 divergence, the hydrodynamic pressure root, the
implicit-function step):

  - Sec. 2.1.2, Eq. (twoFluid cons): per species s (electrons, positrons or
    ions; charge-to-mass ratio mu_s) with primitives (rho_s, v_s, p_s):
    D = sum rho_s W_s, S = sum rho_s h_s W_s^2 v_s + E x B,
    tau = sum (rho_s h_s W_s^2 - p_s - rho_s W_s) + (E^2 + B^2)/2, and the
    mu_s-weighted sums Dbar, Sbar, taubar of the hydrodynamic parts alone;
    psi = phi = 0 at t = 0. There is no Gauss's law step: the charge density
    is Dbar = sum mu_s rho_s W_s.
  - Sec. 2.1.3: primitive recovery. The totals (D, S~ = S - E x B,
    tau~ = tau - (E^2 + B^2)/2) and the weighted sums (Dbar, Sbar, taubar) are
    two linear combinations of the species' hydrodynamic variables, which the
    pair solves for each species; each species then recovers its pressure by
    the single-fluid hydrodynamic root.
  - Appendix A, Eq. (twoFluid flux), (twoFluid source), (twoFluid vars):
    omega_p^2 = sum mu_s^2 rho_s, varrho = sum mu_s rho_s W_s,
    J = sum mu_s rho_s W_s v_s, W = sum mu_s^2 rho_s W_s / omega_p^2,
    u = sum mu_s^2 rho_s W_s v_s / omega_p^2, varrho_0 = W varrho - J.u;
    sources Sbar: omega_p^2 [W E + u x B - eta (J - varrho u)],
    taubar: omega_p^2 [u.E - eta (varrho - varrho_0 W)], E: -J,
    psi: varrho - kappa psi, phi: -kappa phi (eta = 1/sigma), others 0.
  - Sec. 2.2.2 and Tables 1 and 2: as for one fluid (autodiff_sf).
  - Sec. 2.2.1, Eq. (implicit stage): the stiff unknowns of a stage are
    x = (Sbar, taubar, E); D, S, tau, Dbar, B keep their explicit value r;
    psi = (r_psi + a dt r_Dbar) / (1 + a dt kappa) and
    phi = r_phi / (1 + a dt kappa) in closed form (varrho = Dbar has no source);
    x solves G(x) = x - r_x - a dt Psi_x(q(x)) = 0.

Roots (species pressures, stage unknowns) are found on detached values and
joined to the graph by one differentiable Newton step, as in autodiff_sf: at a
converged root that step carries the implicit-function derivative.
"""
from __future__ import annotations

import torch

from .autodiff_sf import (F64, GAMMA_SSP2, _divergence_1d, _pressure_resid, _pressure_root, cross, dot,
                          pad)

# conserved variable order of Sec. 2.1.2
D, S0, TAU, DB, SB0, TAUB, B0, E0, PSI, PHI, NC = 0, 1, 4, 5, 6, 9, 10, 13, 16, 17, 18
# stiff unknowns of an implicit stage: Sbar (3), taubar, E (3)
X_ROWS = (SB0, SB0 + 1, SB0 + 2, TAUB, E0, E0 + 1, E0 + 2)


# ---- Eq. (twoFluid cons) -----------------------------------------------------
def prims_to_cons(P, gamma, mu):
    """P: (16, ...) = (rho_e, v_e, p_e, rho_p, v_p, p_p, B, E); mu = (mu_e, mu_p)."""
    B, E = P[10:13], P[13:16]
    tot = [0.0] * 6  # D, S (3), tau -- hydrodynamic parts
    bar = [0.0] * 6  # Dbar, Sbar (3), taubar
    for s in range(2):
        rho, v, p = P[5 * s], P[5 * s + 1:5 * s + 4], P[5 * s + 4]
        W = 1.0 / torch.sqrt(1.0 - dot(v, v))
        Z = (rho + gamma / (gamma - 1.0) * p) * W * W  # rho h W^2
        parts = [rho * W, Z * v[0], Z * v[1], Z * v[2], Z - p - rho * W]
        for k in range(5):
            tot[k] = tot[k] + parts[k]
            bar[k] = bar[k] + mu[s] * parts[k]
    ExB = cross(E, B)
    z = torch.zeros_like(P[0])
    rows = [tot[0], tot[1] + ExB[0], tot[2] + ExB[1], tot[3] + ExB[2],
            tot[4] + 0.5 * (dot(E, E) + dot(B, B)), bar[0], bar[1], bar[2], bar[3], bar[4]]
    return torch.cat([torch.stack(rows), B, E, z[None], z[None]])


# ---- Sec. 2.1.3: species split and per-species recovery ----------------------
def species_split(q, mu):
    """(D_s, S~_s, tau~_s) of both species from the totals and weighted sums:
    X = X_e + X_p and Xbar = mu_e X_e + mu_p X_p."""
    B, E = q[B0:B0 + 3], q[E0:E0 + 3]
    St = q[S0:S0 + 3] - cross(E, B)
    taut = q[TAU] - 0.5 * (dot(E, E) + dot(B, B))
    me, mp = mu
    tot = (q[D], St, taut)
    bar = (q[DB], q[SB0:SB0 + 3], q[TAUB])
    e = [(xb - mp * x) / (me - mp) for x, xb in zip(tot, bar)]
    p = [(xb - me * x) / (mp - me) for x, xb in zip(tot, bar)]
    return e, p


def recover(q, gamma, mu):
    """Conserved -> per species (rho, v, p, W), differentiable in q through the
    pressure roots' implicit-function derivatives."""
    out = []
    for Ds, Ss, ts in species_split(q, mu):
        St2 = dot(Ss, Ss)
        pd, slope = _pressure_root(Ds, St2, ts, gamma)
        p = pd - _pressure_resid(pd, Ds, St2, ts, gamma) / slope
        v = Ss / (ts + Ds + p)
        W = 1.0 / torch.sqrt(1.0 - dot(v, v))
        out.append((Ds / W, v, p, W))
    return out


def pack(spec):
    """Per-species primitives as one tensor (12, ...): (rho, v, p, W) per species."""
    return torch.cat([torch.cat([r[None], v, p[None], W[None]]) for r, v, p, W in spec])


def unpack(w):
    return [(w[6 * s], w[6 * s + 1:6 * s + 4], w[6 * s + 4], w[6 * s + 5]) for s in range(2)]


# ---- Appendix A: sources and fluxes ------------------------------------------
def auxiliaries(w, mu):
    """(omega_p^2, varrho, J, W, u, varrho_0) of Eq. (twoFluid vars)."""
    wp2 = varrho = Wb = 0.0
    J = u = 0.0
    for s, (rho, v, p, W) in enumerate(unpack(w)):
        wp2 = wp2 + mu[s] ** 2 * rho
        varrho = varrho + mu[s] * rho * W
        J = J + mu[s] * rho * W * v
    for s, (rho, v, p, W) in enumerate(unpack(w)):
        Wb = Wb + mu[s] ** 2 * rho * W / wp2
        u = u + mu[s] ** 2 * rho * W * v / wp2
    varrho0 = Wb * varrho - dot(J, u)
    return wp2, varrho, J, Wb, u, varrho0


def source(q, w, sigma, kappa, mu):
    wp2, varrho, J, Wb, u, varrho0 = auxiliaries(w, mu)
    B, E = q[B0:B0 + 3], q[E0:E0 + 3]
    eta = 1.0 / sigma
    Sb = wp2 * (Wb * E + cross(u, B) - eta * (J - varrho * u))
    tb = wp2 * (dot(u, E) - eta * (varrho - varrho0 * Wb))
    z = torch.zeros_like(q[D])
    rows = [z] * 6 + [Sb[0], Sb[1], Sb[2], tb, z, z, z, -J[0], -J[1], -J[2],
                      varrho - kappa * q[PSI], -kappa * q[PHI]]
    return torch.stack(rows)


def _levi(i, j, k):
    return {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.get((i, j, k), 0)


def flux(q, w, gamma, mu, j):
    """Eq. (twoFluid flux) along direction j."""
    B, E = q[B0:B0 + 3], q[E0:E0 + 3]
    z = torch.zeros_like(q[D])
    fD = fDb = fTb = z
    fS = [z, z, z]
    fSb = [z, z, z]
    for s, (rho, v, p, W) in enumerate(unpack(w)):
        Z = (rho + gamma / (gamma - 1.0) * p) * W * W
        Ds = rho * W
        fD = fD + Ds * v[j]
        fDb = fDb + mu[s] * Ds * v[j]
        for i in range(3):
            Sij = Z * v[i] * v[j] + (p if i == j else 0.0)
            fS[i] = fS[i] + Sij
            fSb[i] = fSb[i] + mu[s] * Sij
        fTb = fTb + (mu[s] * (Z - p - Ds) + mu[s] * p) * v[j]
    em = 0.5 * (dot(E, E) + dot(B, B))
    for i in range(3):
        fS[i] = fS[i] - E[i] * E[j] - B[i] * B[j] + (em if i == j else 0.0)
    fTau = q[S0 + j] - fD
    fB = [sum(_levi(i, j, k) * E[k] for k in range(3)) + (q[PHI] if i == j else 0.0) for i in range(3)]
    fE = [-sum(_levi(i, j, k) * B[k] for k in range(3)) + (q[PSI] if i == j else 0.0) for i in range(3)]
    rows = [fD, *fS, fTau, fDb, *fSb, fTb, *fB, *fE, E[j], B[j]]
    return torch.stack([r if torch.is_tensor(r) else torch.full_like(z, float(r)) for r in rows])


# ---- Sec. 2.2.2: flux divergence (LF splitting + WENO3, as for one fluid) ----
def divergence(q, w, gamma, mu, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    """L(q) for q (18, ny, nx) or (18, nz, ny, nx) with packed primitives w."""
    if q.dim() == 4:  # 3-D
        qg, wg = pad(q, bcx, bcy, bcz), pad(w, bcx, bcy, bcz)
        s_ = slice(2, -2)
        qx, wx = qg[:, s_, s_, :], wg[:, s_, s_, :]
        Lx = _divergence_1d(qx, flux(qx, wx, gamma, mu, 0), dx)
        qy, wy = qg[:, s_, :, s_], wg[:, s_, :, s_]
        Ly = _divergence_1d(qy.transpose(2, 3), flux(qy, wy, gamma, mu, 1).transpose(2, 3), dy).transpose(2, 3)
        qz, wz = qg[:, :, s_, s_], wg[:, :, s_, s_]
        Lz = _divergence_1d(qz.permute(0, 2, 3, 1), flux(qz, wz, gamma, mu, 2).permute(0, 2, 3, 1),
                            dz).permute(0, 3, 1, 2)
        return Lx + Ly + Lz
    qg, wg = pad(q, bcx, bcy), pad(w, bcx, bcy)
    if q.shape[1] == 1:
        return _divergence_1d(qg, flux(qg, wg, gamma, mu, 0), dx)
    qx, wx = qg[:, 2:-2], wg[:, 2:-2]
    Lx = _divergence_1d(qx, flux(qx, wx, gamma, mu, 0), dx)
    qy, wy = qg[:, :, 2:-2], wg[:, :, 2:-2]
    Ly = _divergence_1d(qy.transpose(1, 2), flux(qy, wy, gamma, mu, 1).transpose(1, 2), dy).transpose(1, 2)
    return Lx + Ly


# ---- Sec. 2.2.1: implicit stage ------------------------------------------------
def _stage_q(r, x, adt, kappa):
    ck = 1.0 / (1.0 + adt * kappa)
    rows = list(r.unbind(0))
    for k, v in enumerate(X_ROWS):
        rows[v] = x[k]
    rows[PSI] = (r[PSI] + adt * r[DB]) * ck
    rows[PHI] = r[PHI] * ck
    return torch.stack(rows)


def _stage_G(r, x, adt, sigma, gamma, kappa, mu):
    q = _stage_q(r, x, adt, kappa)
    w = pack(recover(q, gamma, mu))
    s = source(q, w, sigma, kappa, mu)
    idx = torch.tensor(X_ROWS)
    return x - r.index_select(0, idx) - adt * s.index_select(0, idx), q, w


def _admissible(r, x, adt, kappa, mu):
    """Cells whose stage state q(x) leaves each species a pressure root
    (D_s > 0 and |S~_s| < tau~_s + D_s)."""
    q = _stage_q(r, x, adt, kappa)
    good = torch.ones_like(q[D], dtype=torch.bool)
    for Ds, Ss, ts in species_split(q, mu):
        good = good & (Ds > 0) & (ts + Ds > torch.sqrt(dot(Ss, Ss)))
    return good


def _jacobian(r, x, adt, sigma, gamma, kappa, mu):
    """dG/dx per cell, (..., 7, 7), by autograd on detached inputs."""
    xr = x.detach().clone().requires_grad_(True)
    with torch.enable_grad():
        G, _, _ = _stage_G(r.detach(), xr, adt, float(sigma), gamma, kappa, mu)
        rows = [torch.autograd.grad(G[i].sum(), xr, retain_graph=i < 6)[0] for i in range(7)]
    Jm = torch.stack(rows)  # [i][k][cells...] = dG_i/dx_k
    return G.detach(), Jm.movedim(0, -1).movedim(0, -1)


def _solve(Jm, G):
    return torch.linalg.solve(Jm, G.movedim(0, -1).unsqueeze(-1)).squeeze(-1).movedim(-1, 0)


def _newton(rd, x, adt, sigma, gamma, kappa, mu, iters=60):
    """Newton with backtracking on |G|^2 from x (detached values) to a
    round-off fixed point. Returns (x, converged mask)."""
    # round-off scales: the hydrodynamic unknowns (Sbar, taubar) together, E with B
    tiny = torch.full_like(x[0], 1e-300)
    hyd = lambda y: torch.maximum(y[:4].abs().amax(0), tiny)  # noqa: E731
    emb = lambda y: torch.maximum(torch.maximum(y[4:].abs().amax(0), rd[B0:B0 + 3].abs().amax(0)), tiny)  # noqa: E731
    sh, se = hyd(x), emb(x)
    eps = torch.finfo(F64).eps
    conv = torch.zeros_like(x[0], dtype=torch.bool)
    for _ in range(iters):
        G, Jm = _jacobian(rd, x, adt, sigma, gamma, kappa, mu)
        dx = -_solve(Jm, G)
        m0 = (G * G).sum(0)
        t = torch.ones_like(m0)
        ok = torch.zeros_like(m0, dtype=torch.bool)
        with torch.no_grad():
            # a trial whose species admit no pressure root counts as no
            # decrease (it is evaluated at x instead)
            for _ls in range(12):
                xt = x + t * dx
                adm = _admissible(rd, xt, adt, kappa, mu)
                Gt, _, _ = _stage_G(rd, torch.where(adm, xt, x), adt, sigma, gamma, kappa, mu)
                ok = adm & ((Gt * Gt).sum(0) <= (1.0 - 1e-4 * t) * m0)
                if bool(ok.all()):
                    break
                t = torch.where(ok, t, 0.5 * t)
        st = torch.where(ok, t * dx, torch.zeros_like(dx))
        x = x + st
        sh, se = torch.maximum(sh, hyd(x)), torch.maximum(se, emb(x))
        # converged: the accepted step is at round-off, or no step decreases
        # |G| and the full Newton step is tiny (G at its round-off floor)
        small = ok & (st[:4].abs().amax(0) <= 8 * eps * sh) & (st[4:].abs().amax(0) <= 8 * eps * se)
        floor = ~ok & (dx[:4].abs().amax(0) <= 1e-10 * sh) & (dx[4:].abs().amax(0) <= 1e-10 * se)
        conv = conv | small | floor
        if bool(conv.all()):
            break
    return x, conv


def stage(r, adt, sigma, gamma, kappa, mu):
    """q = r + adt Psi(q). The root is found on detached values from x = r_x;
    cells where that fails are solved again by continuation in a dt (the
    stage for adt / 2^m, ..., adt / 2, adt, each from the previous root: the
    final root is the same, only the path to it differs). Then one
    differentiable Newton step joins the root to the graph."""
    rd = r.detach()
    idx = torch.tensor(X_ROWS)
    x0 = rd.index_select(0, idx).clone()
    sigma_f = float(sigma.detach()) if torch.is_tensor(sigma) else float(sigma)
    x, conv = _newton(rd, x0, adt, sigma_f, gamma, kappa, mu)
    if not bool(conv.all()):
        bad = ~conv
        rb, xb, done = rd[:, bad], x0[:, bad], torch.zeros(int(bad.sum()), dtype=torch.bool)
        for m in (3, 6, 9, 12):
            xc, okc = xb.clone(), torch.ones_like(done)
            for k in range(m, -1, -1):
                xc, c = _newton(rb, xc, adt * 2.0 ** -k, sigma_f, gamma, kappa, mu)
                okc = okc & c
            xb = torch.where(~done & okc, xc, xb)
            done = done | okc
            if bool(done.all()):
                break
        if not bool(done.all()):
            raise ArithmeticError("implicit stage: no root found")
        x = x.clone()
        x[:, bad] = xb
    _, Jm = _jacobian(rd, x, adt, sigma_f, gamma, kappa, mu)
    Gd, _, _ = _stage_G(r, x, adt, sigma, gamma, kappa, mu)  # differentiable in r and sigma
    q = _stage_q(r, x - _solve(Jm, Gd), adt, kappa)
    return q, pack(recover(q, gamma, mu))


# ---- Tables 1 and 2: one SSP2(222) or SSP3(332) step -------------------------
def ssp2_step(q, dt, sigma, gamma, kappa, mu, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    g = GAMMA_SSP2
    q1, w1 = stage(q, g * dt, sigma, gamma, kappa, mu)
    L1 = divergence(q1, w1, gamma, mu, bcx, bcy, dx, dy, bcz, dz)
    P1 = source(q1, w1, sigma, kappa, mu)
    q2, w2 = stage(q + dt * L1 + (1.0 - 2.0 * g) * dt * P1, g * dt, sigma, gamma, kappa, mu)
    L2 = divergence(q2, w2, gamma, mu, bcx, bcy, dx, dy, bcz, dz)
    P2 = source(q2, w2, sigma, kappa, mu)
    return q + 0.5 * dt * (L1 + L2) + 0.5 * dt * (P1 + P2)


def ssp3_step(q, dt, sigma, gamma, kappa, mu, bcx, bcy, dx, dy, bcz=1, dz=1.0):
    g = GAMMA_SSP2
    q1, w1 = stage(q, g * dt, sigma, gamma, kappa, mu)
    L1 = divergence(q1, w1, gamma, mu, bcx, bcy, dx, dy, bcz, dz)
    P1 = source(q1, w1, sigma, kappa, mu)
    q2, w2 = stage(q + dt * L1 + (1.0 - 2.0 * g) * dt * P1, g * dt, sigma, gamma, kappa, mu)
    L2 = divergence(q2, w2, gamma, mu, bcx, bcy, dx, dy, bcz, dz)
    P2 = source(q2, w2, sigma, kappa, mu)
    q3, w3 = stage(q + 0.25 * dt * (L1 + L2) + (0.5 - g) * dt * P1, g * dt, sigma, gamma, kappa, mu)
    L3 = divergence(q3, w3, gamma, mu, bcx, bcy, dx, dy, bcz, dz)
    P3 = source(q3, w3, sigma, kappa, mu)
    return q + dt / 6.0 * (L1 + P1) + dt / 6.0 * (L2 + P2) + 2.0 * dt / 3.0 * (L3 + P3)


def run(prims, sigma, dt, nsteps, gamma, mu, bcx, bcy, dx, dy, kappa=1.0, scheme=0, bcz=1, dz=1.0):
    """prims (16, ny, nx), or (16, nz, ny, nx), and sigma (0-d) as tensors (may
    require grad) -> q^n; mu = (mu_e, mu_p); scheme 0: SSP2(222), 1: SSP3(332)."""
    step = ssp3_step if scheme == 1 else ssp2_step
    q = prims_to_cons(prims, gamma, mu)
    for _ in range(nsteps):
        q = step(q, dt, sigma, gamma, kappa, mu, bcx, bcy, dx, dy, bcz, dz)
    return q


def gradient(wl, nsteps, lam, scheme=0, prims=None):
    """J = sum(lam * q^n) for a two-fluid workload (fields name, prims, sigma,
    gamma, mu_e, mu_p, kappa, bc_x, bc_y, bc_z, dx, dy, dz, nz, cfl):
    returns (J, dJ/dprims, dJ/dsigma, q^n) as NumPy/float."""
    P = torch.tensor(wl.prims if prims is None else prims, dtype=F64, requires_grad=True)
    s = torch.tensor(float(wl.sigma), dtype=F64, requires_grad=True)
    q = run(P, s, wl.dt, nsteps, wl.gamma, (wl.mu_e, wl.mu_p), wl.bc_x, wl.bc_y, wl.dx, wl.dy, wl.kappa, scheme,
            wl.bc_z, wl.dz)
    J = (torch.tensor(lam, dtype=F64) * q).sum()
    gP, gs = torch.autograd.grad(J, (P, s))
    return float(J.detach()), gP.numpy(), float(gs), q.detach().numpy()


def forward(wl, nsteps, scheme=0, prims=None, sigma=None):
    """q^n of a two-fluid workload without a graph."""
    with torch.no_grad():
        P = torch.tensor(wl.prims if prims is None else prims, dtype=F64)
        s = torch.tensor(float(wl.sigma if sigma is None else sigma), dtype=F64)
        return run(P, s, wl.dt, nsteps, wl.gamma, (wl.mu_e, wl.mu_p), wl.bc_x, wl.bc_y, wl.dx, wl.dy, wl.kappa,
                   scheme, wl.bc_z, wl.dz).numpy()


def jvp(wl, nsteps, v_prims, v_sigma, scheme=0):
    """Directional derivative of q^n along (v_prims, v_sigma): reverse mode
    applied twice. g(u) = d<u, q^n>/d(prims, sigma) is linear in u, so the
    derivative of <g(u), v> with respect to u is J v at any u."""
    P = torch.tensor(wl.prims, dtype=F64, requires_grad=True)
    s = torch.tensor(float(wl.sigma), dtype=F64, requires_grad=True)
    q = run(P, s, wl.dt, nsteps, wl.gamma, (wl.mu_e, wl.mu_p), wl.bc_x, wl.bc_y, wl.dx, wl.dy, wl.kappa, scheme,
            wl.bc_z, wl.dz)
    u = torch.zeros_like(q, requires_grad=True)
    gP, gs = torch.autograd.grad((u * q).sum(), (P, s), create_graph=True)
    inner = (gP * torch.tensor(v_prims, dtype=F64)).sum() + gs * float(v_sigma)
    (Jv,) = torch.autograd.grad(inner, u)
    return Jv.numpy()
