"""Sedov-Taylor self-similar point blast (spherical, ideal gas).

TEST INFRASTRUCTURE: a reference solution that pins the oracle's 3-D runs.

Derivation used here (written out from the Euler equations, not from a
table): with the shock radius R(t) = xi0 (E t^2 / rho0)^(1/5) and
Rdot = 2R/(5t), look for u = Rdot phi(xi), rho = rho0 psi(xi),
p = rho0 Rdot^2 pi(xi), xi = r/R.  Mass, momentum and entropy conservation
in spherical symmetry reduce to three ODEs in xi:

    (phi - xi) psi' + psi phi'  = -2 psi phi / xi
    (phi - xi) phi' + pi'/psi   =  3/2 phi
    (phi - xi) (pi'/pi - gamma psi'/psi) = 3

(the 3/2 and 3 come from Rddot = -3/2 Rdot^2 / R for R ~ t^(2/5)), with the
strong-shock jump conditions at xi = 1:
    phi = 2/(gamma+1),  psi = (gamma+1)/(gamma-1),  pi = 2/(gamma+1).
The blast energy E = 4 pi rho0 Rdot^2 R^3 I with
    I = int_0^1 (psi phi^2 / 2 + pi/(gamma-1)) xi^2 dxi
and Rdot^2 R^3 = (4/25) xi0^5 E / rho0 gives xi0^5 = 25 / (16 pi I).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(xi, y, gamma):
    phi, psi, pi = y
    a = phi - xi
    # rows: continuity, momentum, entropy; unknowns (phi', psi', pi')
    M = np.array([
        [psi, a, 0.0],
        [a, 0.0, 1.0 / psi],
        [0.0, -a * gamma / psi, a / pi],
    ])
    b = np.array([-2.0 * psi * phi / xi, 1.5 * phi, 3.0])
    return np.linalg.solve(M, b)


def profile(gamma=1.4, xi_min=1e-3, npts=4000):
    """Self-similar profile on xi in [xi_min, 1]: (xi, phi, psi, pi)."""
    y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
    xs = np.linspace(1.0, xi_min, npts)
    sol = solve_ivp(_rhs, (1.0, xi_min), y0, t_eval=xs, args=(gamma,), method="LSODA",
                    rtol=1e-11, atol=1e-14)
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.t[::-1], sol.y[0][::-1], sol.y[1][::-1], sol.y[2][::-1]


def energy_integral(gamma=1.4):
    xi, phi, psi, pi = profile(gamma)
    integrand = (0.5 * psi * phi ** 2 + pi / (gamma - 1.0)) * xi ** 2
    return float(np.trapezoid(integrand, xi))


def xi0(gamma=1.4):
    """Dimensionless constant of R(t) = xi0 (E t^2/rho0)^(1/5)."""
    return (25.0 / (16.0 * math.pi * energy_integral(gamma))) ** 0.2


def shock_radius(t, energy=1.0, rho0=1.0, gamma=1.4):
    return xi0(gamma) * (energy * t * t / rho0) ** 0.2
