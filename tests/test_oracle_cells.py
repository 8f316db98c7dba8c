"""Pins of the CPU oracle's per-cell pieces against hand-worked closed forms and
invariants (no GPU). Each pin is chosen so that a dropped term, a wrong sign or
a swapped index in the oracle fails it.

Paper: Wright & Hawke, arXiv:1808.09721 -- Sec. 2.1.1 (one fluid), Sec. 2.1.2 and
Appendix A (two fluids), Sec. 2.1.3 (primitive recovery), Sec. 2.2.2 (WENO3).
"""
import math

import numpy as np
import pytest

import oracle as O
from conftest import load_golden
from paper_1808_09721_gb300 import workloads as WL


def _close(a, b, rtol=1e-14, atol=1e-14):
    np.testing.assert_allclose(np.asarray(a), np.asarray(b), rtol=rtol, atol=atol)


# ---------------------------------------------------------------- single fluid
def test_sf_hand_worked_cell():
    """Eq. (resistive prims) + Eq. (resistive RMHD) on a hand-worked state."""
    g = load_golden("sf_cell.txt")
    varrho, psi, phi, gamma, sigma, kappa = g["extra"]
    q = O.sf_p2c(g["prim"], varrho, psi, phi, gamma)
    _close(q, g["cons"])
    w = O.sf_c2p(q, gamma)
    _close(w, g["prim"][:5], rtol=1e-13, atol=1e-13)
    _close(O.sf_flux(q, w, gamma, sigma, 0), g["flux_x"], rtol=1e-13, atol=1e-13)
    _close(O.sf_flux(q, w, gamma, sigma, 1), g["flux_y"], rtol=1e-13, atol=1e-13)
    _close(O.sf_source(q, w, sigma, kappa), g["source"], rtol=1e-13, atol=1e-13)
    _close(O.sf_current(q, w, sigma), g["current"], rtol=1e-13, atol=1e-13)


def test_sf_ohm_parallel_term():
    """J = W sigma [E - (v.E) v] for E parallel to v, B = 0, varrho = 0:
    v = (0.6,0,0), E = (1,0,0), sigma = 1 -> J = 1.25 * (1 - 0.36) = 0.8 along x."""
    q = O.sf_p2c([1, 0.6, 0, 0, 1, 0, 0, 0, 1, 0, 0], 0.0, 0.0, 0.0, 2.0)
    w = O.sf_c2p(q, 2.0)
    _close(O.sf_current(q, w, 1.0), [0.8, 0.0, 0.0], rtol=1e-14, atol=1e-14)


def test_sf_round_trip_random():
    """prims -> cons -> prims to 1e-12 relative over W in [1, 10], p/rho in [1e-2, 1e2],
    |E|, |B| <= 1 (Sec. 2.1.3; the recovery is the inverse of Eq. (resistive prims)).
    The recovery's condition number grows like W^2, so the bound is
    max(1e-12, 2e-14 W^2) relative (1e-12 up to W = 7, 2e-12 at W = 10)."""
    states = WL.random_sf_states(400, seed=11)
    for gamma in (4.0 / 3.0, 5.0 / 3.0, 2.0):
        for s in states:
            q = O.sf_p2c(s, 0.0, 0.0, 0.0, gamma)
            w = O.sf_c2p(q, gamma)
            W2 = 1.0 / (1.0 - np.dot(s[1:4], s[1:4]))
            tol = max(1e-12, 2e-14 * W2)
            assert abs(w[0] - s[0]) <= tol * s[0]
            assert abs(w[4] - s[4]) <= tol * s[4]
            assert np.max(np.abs(w[1:4] - s[1:4])) <= 1e-12


def test_sf_round_trip_wide_range():
    """Wider states (W up to 10, p/rho in [1e-3, 1e3], |E|, |B| up to 10): the
    recovered pressure agrees to 1e-12 of the cell's energy scale tau + D."""
    states = WL.random_sf_states(300, seed=12, theta=(1e-3, 1e3), emax=10.0, bmax=10.0)
    for s in states:
        q = O.sf_p2c(s, 0.0, 0.0, 0.0, 4.0 / 3.0)
        w = O.sf_c2p(q, 4.0 / 3.0)
        scale = q[4] + q[0]
        assert abs(w[4] - s[4]) <= 1e-12 * scale
        assert np.max(np.abs(w[1:4] - s[1:4])) <= 1e-11


def test_c2p_rejects_unphysical():
    """|S~| >= tau~ + D has no admissible root: the recovery reports failure."""
    with pytest.raises(O.OracleError):
        O.hydro_c2p(1.0, [5.0, 0.0, 0.0], 1.0, 4.0 / 3.0)
    with pytest.raises(O.OracleError):
        O.hydro_c2p(-1.0, [0.0, 0.0, 0.0], 1.0, 4.0 / 3.0)


def test_c2p_rest_frame_closed_form():
    """At rest (S~ = 0): W = 1, rho = D and tau~ = rho eps = p/(Gamma-1), so
    p = (Gamma - 1) tau~ exactly (Gamma-law EOS, Sec. 2.1). The root is found to
    round-off of the residual's largest term, i.e. a few ulp of tau~ + D."""
    for gamma in (4.0 / 3.0, 5.0 / 3.0, 2.0):
        for D, taut in ((1.0, 3.0), (0.125, 0.25), (10.0, 1e-3)):
            w = O.hydro_c2p(D, [0.0, 0.0, 0.0], taut, gamma)
            _close(w, [D, 0.0, 0.0, 0.0, (gamma - 1.0) * taut], rtol=1e-14,
                   atol=8 * np.finfo(float).eps * (taut + D))


# ---------------------------------------------------------------- two fluids
def test_tf_hand_worked_cell():
    """Eq. (twoFluid cons), Appendix A flux and source on a hand-worked state with
    unequal charge-to-mass ratios (mu_e = -2, mu_p = 3) so species swaps show."""
    g = load_golden("tf_cell.txt")
    mu_e, mu_p, gamma, sigma, kappa, psi, phi = g["extra"]
    q = O.tf_p2c(g["prim"], gamma, mu_e, mu_p, psi, phi)
    _close(q, g["cons"], rtol=1e-14, atol=1e-14)
    w = O.tf_c2p(q, gamma, mu_e, mu_p)
    _close(w, g["prim"][:10], rtol=1e-12, atol=1e-12)
    _close(O.tf_flux(q, w, gamma, mu_e, mu_p, 0), g["flux_x"], rtol=1e-12, atol=1e-12)
    _close(O.tf_flux(q, w, gamma, mu_e, mu_p, 1), g["flux_y"], rtol=1e-12, atol=1e-12)
    _close(O.tf_source(q, w, sigma, mu_e, mu_p, kappa), g["source"], rtol=1e-12, atol=1e-12)


def test_tf_round_trip_random():
    """Species decomposition (Sec. 2.1.3) + per-species recovery invert Eq. (twoFluid cons)."""
    states = WL.random_tf_states(300, seed=13)
    for mu_e, mu_p in ((-1e3, 1e3), (-1e5, 1e3), (-2.0, 3.0)):
        for s in states:
            q = O.tf_p2c(s, 4.0 / 3.0, mu_e, mu_p)
            w = O.tf_c2p(q, 4.0 / 3.0, mu_e, mu_p)
            for k in (0, 5):
                scale = q[0] + q[4]
                assert abs(w[k] - s[k]) <= 1e-10 * scale
                assert abs(w[k + 4] - s[k + 4]) <= 1e-10 * scale
                assert np.max(np.abs(w[k + 1:k + 4] - s[k + 1:k + 4])) <= 1e-9


def test_tf_neutral_pair_has_no_charge_or_current():
    """mu_p = -mu_e with identical species: varrho = 0, J = 0, so the E and psi
    sources vanish (Appendix A auxiliaries), and Dbar = Sbar = taubar = 0."""
    s = np.array([0.7, 0.3, -0.2, 0.1, 0.9] * 2 + [0.2, 0.5, -0.1, 0.05, 0.0, 0.3])
    q = O.tf_p2c(s, 4.0 / 3.0, -1e3, 1e3)
    assert np.all(np.abs(q[5:10]) <= 1e-12)
    w = O.tf_c2p(q, 4.0 / 3.0, -1e3, 1e3)
    src = O.tf_source(q, w, 1e4, -1e3, 1e3, kappa=1.0)
    assert np.all(np.abs(src[13:16]) <= 1e-9)     # -J
    assert abs(src[16]) <= 1e-9                   # varrho - kappa psi with psi = 0


def test_tf_reduces_to_one_fluid_sums():
    """With identical species the two-fluid totals (D, S, tau) equal the one-fluid
    conserved values of the summed density and pressure at the same velocity."""
    sp = [0.4, 0.3, 0.0, -0.2, 0.5]
    E, B = [0.1, -0.2, 0.3], [0.4, 0.1, -0.5]
    qt = O.tf_p2c(sp + sp + B + E, 5.0 / 3.0, -7.0, 9.0)
    qs = O.sf_p2c([0.8, 0.3, 0.0, -0.2, 1.0] + B + E, 0.0, 0.0, 0.0, 5.0 / 3.0)
    _close(qt[0:5], qs[0:5], rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- WENO3
def test_weno3_constant_and_linear_exact():
    """WENO3 (Sec. 2.2.2) reproduces constant and linear data at the face exactly:
    both candidate polynomials are exact, so any convex weights are."""
    assert O.weno3(2.5, 2.5, 2.5) == 2.5
    for a, b in ((1.0, 0.5), (-3.0, 2.0), (0.1, -0.01)):
        got = O.weno3(a - b, a, a + b)
        assert abs(got - (a + 0.5 * b)) <= 1e-15 * (abs(a) + abs(b))


def test_weno3_linear_weights_on_symmetric_data():
    """Equal smoothness indicators give the linear weights (1/3, 2/3):
    fhat = -f_{i-1}/6 + 5 f_i/6 + f_{i+1}/3; for (1, 0, 1) this is 1/6."""
    assert abs(O.weno3(1.0, 0.0, 1.0) - 1.0 / 6.0) <= 1e-15
    assert abs(O.weno3(-2.0, 1.0, 4.0) - (2.0 / 6 + 5.0 / 6 + 4.0 / 3)) <= 1e-14


def test_weno3_picks_smooth_stencil_at_jump():
    """At a jump on the right the left stencil (weight ~1) is used: (0, 0, 1) -> ~0;
    a jump on the left uses the central stencil: (1, 0, 0) -> ~0."""
    assert abs(O.weno3(0.0, 0.0, 1.0)) <= 1e-11
    assert abs(O.weno3(1.0, 0.0, 0.0)) <= 1e-11
    assert abs(O.weno3(0.0, 1.0, 1.0) - 1.0) <= 1e-11
