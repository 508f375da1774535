"""Exact solution of the 1-D Riemann problem for the ideal-gas Euler equations.

TEST INFRASTRUCTURE: a reference solution that pins the oracle (shock-tube
test).  Written from the theory of the exact Riemann solver (Toro, Riemann
Solvers and Numerical Methods for Fluid Dynamics, Ch. 4): the star pressure
p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic
Riemann-invariant) branch for p <= p_K; u* follows from the same functions.
The wave pattern is then sampled on x/t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class StarState:
    p: float
    u: float
    rho_L: float
    rho_R: float
    shock_speed_R: float | None
    shock_speed_L: float | None


def _f_and_df(p, rho, pk, gamma):
    """Velocity jump across the wave connecting p_K to p, and its derivative."""
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        e = (gamma - 1.0) / (2.0 * gamma)
        f = 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-15):
    """left/right = (rho, u, p).  Newton iteration on the pressure function."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    if 2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    # two-rarefaction guess
    e = (gamma - 1.0) / (2.0 * gamma)
    p = ((cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)) / (cl / pl ** e + cr / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(100):
        fl, dfl = _f_and_df(p, rl, pl, gamma)
        fr, dfr = _f_and_df(p, rr, pr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, gamma)
    fr, _ = _f_and_df(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if p > pl:
        rho_l = rl * (p / pl + g1) / (g1 * p / pl + 1.0)
        sl = ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * p / pl + (gamma - 1.0) / (2.0 * gamma))
    else:
        rho_l = rl * (p / pl) ** (1.0 / gamma)
        sl = None
    if p > pr:
        rho_r = rr * (p / pr + g1) / (g1 * p / pr + 1.0)
        sr = ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * p / pr + (gamma - 1.0) / (2.0 * gamma))
    else:
        rho_r = rr * (p / pr) ** (1.0 / gamma)
        sr = None
    return StarState(p, u, rho_l, rho_r, sr, sl)


def sample(left, right, s, gamma=1.4):
    """(rho, u, p) of the self-similar solution at x/t = s (scalar or array)."""
    st = star_state(left, right, gamma)
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    g = gamma
    for n, x in enumerate(s):
        if x <= st.u:  # left of the contact
            if st.p > pl:  # left shock
                if x <= st.shock_speed_L:
                    rho[n], u[n], p[n] = rl, ul, pl
                else:
                    rho[n], u[n], p[n] = st.rho_L, st.u, st.p
            else:  # left rarefaction
                c_star = cl * (st.p / pl) ** ((g - 1.0) / (2.0 * g))
                head, tail = ul - cl, st.u - c_star
                if x <= head:
                    rho[n], u[n], p[n] = rl, ul, pl
                elif x >= tail:
                    rho[n], u[n], p[n] = st.rho_L, st.u, st.p
                else:
                    fac = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cl) * (ul - x)
                    rho[n] = rl * fac ** (2.0 / (g - 1.0))
                    u[n] = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + x)
                    p[n] = pl * fac ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if st.p > pr:  # right shock
                if x >= st.shock_speed_R:
                    rho[n], u[n], p[n] = rr, ur, pr
                else:
                    rho[n], u[n], p[n] = st.rho_R, st.u, st.p
            else:  # right rarefaction
                c_star = cr * (st.p / pr) ** ((g - 1.0) / (2.0 * g))
                head, tail = ur + cr, st.u + c_star
                if x >= head:
                    rho[n], u[n], p[n] = rr, ur, pr
                elif x <= tail:
                    rho[n], u[n], p[n] = st.rho_R, st.u, st.p
                else:
                    fac = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * cr) * (ur - x)
                    rho[n] = rr * fac ** (2.0 / (g - 1.0))
                    u[n] = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + x)
                    p[n] = pr * fac ** (2.0 * g / (g - 1.0))
    return rho, u, p


def cell_average_density(left, right, x_faces, x0, t, gamma=1.4, sub=64):
    """Cell averages of the exact density over cells [x_faces[i], x_faces[i+1]]."""
    x_faces = np.asarray(x_faces, dtype=np.float64)
    out = np.empty(len(x_faces) - 1)
    for i in range(len(out)):
        xs = x_faces[i] + (np.arange(sub) + 0.5) / sub * (x_faces[i + 1] - x_faces[i])
        rho, _, _ = sample(left, right, (xs - x0) / t, gamma)
        out[i] = rho.mean()
    return out
