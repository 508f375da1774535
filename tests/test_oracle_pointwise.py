"""Pins of the oracle's pointwise arithmetic (EOS, MC limiter, HLLC).

Each check compares against something other than the oracle's own formula:
definitions evaluated by hand, exact special cases of the Riemann problem,
symmetries, and the jump / consistency relations an HLLC fan must satisfy.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
import workloads as wl

G = 1.4


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------- EOS -------

def test_prim_roundtrip_of_stated_state():
    # conserved data built from a stated primitive state (input definition)
    W = (1.3, 0.4, -0.7, 0.2, 2.1)
    U = wl.conserved(*[np.array(x) for x in W], G)
    w, hit = orc.prim(U.ravel())
    assert hit == 0
    assert rel(w, W) < 4e-16


def test_prim_floors_counted():
    U = wl.conserved(np.array(1.0), 0.0, 0.0, 0.0, -1.0, G).ravel()  # negative pressure
    w, hit = orc.prim(U)
    assert hit == 1 and w[4] == 1e-14
    w, hit = orc.prim(np.array([1e-20, 0, 0, 0, 1.0]))
    assert hit == 1 and w[0] == 1e-12


# ------------------------------------------------------------ MC limiter ----

@pytest.mark.parametrize("qm,q0,qp,expect", [
    (1.0, 2.0, 1.0, 0.0),        # extremum: opposite signs
    (1.0, 1.0, 3.0, 0.0),        # one-sided difference exactly zero
    (0.0, 1.0, 2.0, 1.0),        # equal differences: central slope
    (0.0, 1.0, 5.0, 2.0),        # 4 dm < dp: capped at 2 dm
    (0.0, 4.0, 5.0, 2.0),        # dm > 4 dp: capped at 2 dp
    (0.0, 1.0, 2.5, 1.25),       # central (dm+dp)/2 smallest
    (5.0, 4.0, 0.0, -2.0),       # decreasing: negative sign
    (2.0, 1.0, 0.0, -1.0),
])
def test_mc_hand_cases(qm, q0, qp, expect):
    assert orc.mc_slope(qm, q0, qp) == expect


def test_mc_face_values_bounded_by_neighbours():
    rng = np.random.default_rng(3)
    q = rng.normal(size=(20000, 3))
    for qm, q0, qp in q:
        s = orc.mc_slope(qm, q0, qp)
        lo, hi = min(qm, q0, qp), max(qm, q0, qp)
        for face in (q0 - 0.5 * s, q0 + 0.5 * s):
            assert lo - 1e-15 <= face <= hi + 1e-15


# ------------------------------------------------------------------ HLLC ----

def euler_flux_by_definition(W):
    """F(U) of the Euler equations, written directly from the conservation law."""
    r, u, v, w, p = W
    E = p / (G - 1) + 0.5 * r * (u * u + v * v + w * w)
    return np.array([r * u, r * u * u + p, r * u * v, r * u * w, (E + p) * u])


def random_states(n, seed, mach=2.0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = rng.uniform(0.1, 3.0)
        p = rng.uniform(0.05, 3.0)
        c = math.sqrt(G * p / r)
        vel = rng.uniform(-mach, mach, 3) * c
        out.append(np.array([r, *vel, p]))
    return out


def test_hllc_consistency_equal_states():
    for W in random_states(200, 1):
        F = orc.hllc(W, W)
        assert rel(F, euler_flux_by_definition(W)) < 2e-14


def test_hllc_supersonic_is_upwind():
    for W in random_states(100, 2, mach=0.5):
        WL = W.copy(); WR = W.copy()
        c = math.sqrt(G * W[4] / W[0])
        WL[1] = 3.0 * c
        WR[1] = 3.5 * c
        WR[0] *= 1.1
        WR[4] *= 0.9
        F, d = orc.hllc(WL, WR, detail=True)
        assert d["region"] == 0
        assert rel(F, euler_flux_by_definition(WL)) < 1e-15
        F, d = orc.hllc(WR * np.array([1, -1, 1, 1, 1]), WL * np.array([1, -1, 1, 1, 1]), detail=True)
        assert d["region"] == 3


def test_hllc_stationary_contact_exact():
    # pressure and normal velocity continuous, density and tangential velocity jump
    WL = np.array([1.0, 0.0, 0.3, -0.1, 0.7])
    WR = np.array([0.2, 0.0, -0.5, 0.4, 0.7])
    F, d = orc.hllc(WL, WR, detail=True)
    assert d["Ss"] == 0.0
    assert np.allclose(F, [0.0, 0.7, 0.0, 0.0, 0.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("u0", [0.37, -0.52])
def test_hllc_moving_contact_exact(u0):
    WL = np.array([1.0, u0, 0.2, 0.0, 0.9])
    WR = np.array([0.3, u0, -0.4, 0.1, 0.9])
    F, d = orc.hllc(WL, WR, detail=True)
    assert abs(d["Ss"] - u0) < 1e-15
    up = WL if u0 > 0 else WR
    assert rel(F, euler_flux_by_definition(up)) < 1e-14


def test_hllc_mirror_symmetry():
    M = np.array([1, -1, 1, 1, 1.0])
    flip = np.array([-1, 1, -1, -1, -1.0])  # mass, tangential momenta and energy fluxes change sign
    for a, b in zip(random_states(100, 4), random_states(100, 5)):
        F = orc.hllc(a, b)
        Fm = orc.hllc(b * M, a * M)
        assert np.max(np.abs(F - flip * Fm)) <= 1e-13 * max(1.0, np.max(np.abs(F)))


def test_hllc_fan_relations():
    """Relations that hold for the HLLC fan whatever the states:
    - wave-speed bounds S_L <= u_L - c_L, S_R >= u_R + c_R, S_L < S* < S_R;
    - star states carry the contact speed: (rho u)*_K = S* rho*_K;
    - Rankine-Hugoniot across the contact: F*_R - F*_L = S* (U*_R - U*_L);
    - integral consistency of the fan:
      (S* - S_L) U*_L + (S_R - S*) U*_R = S_R U_R - S_L U_L - (F_R - F_L);
    - the returned flux is the one of the region that contains x/t = 0."""
    for a, b in zip(random_states(300, 6), random_states(300, 7)):
        F, d = orc.hllc(a, b, detail=True)
        cL = math.sqrt(G * a[4] / a[0]); cR = math.sqrt(G * b[4] / b[0])
        SL, SR, Ss = d["SL"], d["SR"], d["Ss"]
        assert SL <= a[1] - cL + 1e-14 and SR >= b[1] + cR - 1e-14
        assert SL < Ss < SR
        for k in ("UsL", "UsR"):
            assert abs(d[k][1] - Ss * d[k][0]) <= 1e-13 * max(1.0, abs(d[k][1]))
        lhs = d["FsR"] - d["FsL"]
        rhs = Ss * (d["UsR"] - d["UsL"])
        scale = max(1.0, np.max(np.abs(d["FsL"])), np.max(np.abs(d["FsR"])))
        assert np.max(np.abs(lhs - rhs)) <= 1e-12 * scale
        lhs = (Ss - SL) * d["UsL"] + (SR - Ss) * d["UsR"]
        rhs = SR * d["UR"] - SL * d["UL"] - (d["FR"] - d["FL"])
        scale = max(1.0, np.max(np.abs(SR * d["UR"])), np.max(np.abs(SL * d["UL"])))
        assert np.max(np.abs(lhs - rhs)) <= 1e-12 * scale
        assert rel(d["FL"], euler_flux_by_definition(a)) < 1e-14
        assert rel(d["FR"], euler_flux_by_definition(b)) < 1e-14
        region = 0 if SL >= 0 else (1 if Ss >= 0 else (2 if SR > 0 else 3))
        assert d["region"] == region
        expect = [d["FL"], d["FsL"], d["FsR"], d["FR"]][region]
        assert np.array_equal(F, expect)


def test_hllc_sod_face_star_pressure_bracketed():
    """At the initial Sod face the HLLC contact speed lies between the two
    acoustic bounds and the mass flux is positive (flow to the right), as the
    exact solution (u* = 0.927 > 0) requires."""
    F, d = orc.hllc(np.array([1.0, 0, 0, 0, 1.0]), np.array([0.125, 0, 0, 0, 0.1]), detail=True)
    assert d["Ss"] > 0 and F[0] > 0
    assert d["SL"] <= -math.sqrt(1.4) + 1e-15
    assert d["SR"] >= math.sqrt(1.4 * 0.1 / 0.125) - 1e-15


def test_hllc_sod_face_in_50_digit_arithmetic():
    """The initial Sod face worked through in 50-digit decimal arithmetic, step
    by step from the definitions (Roe averages with sqrt(rho) weights, Einfeldt
    bounds, Toro's contact speed and left star state; the fan straddles the
    face with S* > 0, so F = F_L + S_L (U*_L - U_L)).  The oracle's double
    result agrees to rounding: a check of its evaluation order and constants
    at one stated face, beside the structural pins above."""
    from decimal import Decimal as D, getcontext
    getcontext().prec = 50
    g = D("1.4")
    rL, pL, rR, pR = D(1), D(1), D("0.125"), D("0.1")
    EL, ER = pL / (g - 1), pR / (g - 1)                 # at rest: E = p / (gamma - 1)
    cL, cR = (g * pL / rL).sqrt(), (g * pR / rR).sqrt()
    r = rR.sqrt() / rL.sqrt()
    ut = D(0)                                          # (u_L + r u_R) / (1 + r) with u = 0
    HL, HR = (EL + pL) / rL, (ER + pR) / rR            # 3.5 and 2.8
    Ht = (HL + r * HR) / (1 + r)
    ct = ((g - 1) * (Ht - ut * ut / 2)).sqrt()
    SL, SR = min(-cL, ut - ct), max(cR, ut + ct)
    Ss = (pR - pL) / (rL * SL - rR * SR)               # Toro's contact speed with u_L = u_R = 0
    assert Ss > 0 and SL < 0
    k = rL * SL / (SL - Ss)                            # rho_L (S_L - u_L) / (S_L - S*)
    Ustar = [k, k * Ss, D(0), D(0), k * (EL / rL + Ss * (Ss + pL / (rL * SL)))]
    UL = [rL, D(0), D(0), D(0), EL]
    FL = [D(0), pL, D(0), D(0), D(0)]
    F = [FL[i] + SL * (Ustar[i] - UL[i]) for i in range(5)]
    Fo, d = orc.hllc(np.array([1.0, 0, 0, 0, 1.0]), np.array([0.125, 0, 0, 0, 0.1]), detail=True)
    scale = max(abs(float(x)) for x in F)
    assert max(abs(Fo[i] - float(F[i])) for i in range(5)) <= 1e-15 * scale
    for key, ref in (("SL", SL), ("SR", SR), ("Ss", Ss)):
        assert abs(d[key] - float(ref)) <= 1e-15 * abs(float(ref))
    assert Fo[2] == 0.0 and Fo[3] == 0.0


def test_euler_flux_entry_point():
    for W in random_states(50, 9):
        assert rel(orc.euler_flux(W), euler_flux_by_definition(W)) < 1e-15
