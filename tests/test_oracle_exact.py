"""Pins of the exact reference solutions used to pin the oracle's runs."""
import json
import math
import os

import numpy as np

from oracle import exact_riemann as er
from oracle import sedov

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_sod_star_state_matches_tabulated_values():
    g = load("sod_star_state.json")
    st = er.star_state(tuple(g["left"]), tuple(g["right"]), g["gamma"])
    tol = 0.5 * 10 ** (-(g["digits"] - 1))
    for got, key in [(st.p, "p_star"), (st.u, "u_star"), (st.rho_L, "rho_star_left"),
                     (st.rho_R, "rho_star_right"), (st.shock_speed_R, "shock_speed")]:
        assert abs(got - g[key]) <= tol * abs(g[key]), key


def test_exact_riemann_rankine_hugoniot_across_shock():
    """Mass, momentum and energy fluxes in the shock frame agree on both sides."""
    G = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    st = er.star_state(left, right, G)
    s = st.shock_speed_R
    r1, u1, p1 = right
    r2, u2, p2 = st.rho_R, st.u, st.p
    def fluxes(r, u, p):
        w = u - s
        E = p / (G - 1) + 0.5 * r * w * w
        return np.array([r * w, r * w * w + p, w * (E + p)])
    a, b = fluxes(r1, u1, p1), fluxes(r2, u2, p2)
    assert np.max(np.abs(a - b)) < 1e-12


def test_exact_riemann_isentropic_rarefaction():
    """p/rho^gamma is constant through the left rarefaction, and u + 2c/(g-1) too."""
    G = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    s = np.linspace(-1.1, -0.1, 50)
    rho, u, p = er.sample(left, right, s, G)
    ent = p / rho ** G
    inv = u + 2 * np.sqrt(G * p / rho) / (G - 1)
    assert np.ptp(ent) < 1e-13 and np.ptp(inv) < 1e-13


def test_exact_riemann_symmetric_problem():
    """Colliding symmetric streams: u* = 0 and equal star densities."""
    st = er.star_state((1.0, 1.0, 1.0), (1.0, -1.0, 1.0))
    assert abs(st.u) < 1e-14 and abs(st.rho_L - st.rho_R) < 1e-13


def test_sedov_xi0_matches_tabulated():
    g = load("sedov_xi0.json")
    for case in g["cases"]:
        assert abs(sedov.xi0(case["gamma"]) - case["xi0"]) <= g["abs_tol"]


def test_sedov_profile_jump_and_centre():
    """Shock values at xi=1 are the strong-shock limits, pressure tends to a
    finite central value and the density vanishes at the centre."""
    G = 1.4
    xi, phi, psi, pi = sedov.profile(G)
    assert abs(psi[-1] - (G + 1) / (G - 1)) < 1e-12
    assert abs(phi[-1] - 2 / (G + 1)) < 1e-12
    assert psi[0] < 1e-3 * psi[-1]
    assert 0.2 < pi[0] / pi[-1] < 0.5
    # velocity is monotone and roughly linear near the centre (phi/xi -> const)
    r = phi[:50] / xi[:50]
    assert np.ptp(r) < 0.01 * r.mean()
