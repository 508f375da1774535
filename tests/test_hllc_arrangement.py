"""The HLLC arrangement the CUDA path evaluates, against the oracle's HLLC.

The oracle computes the HLLC flux with Einfeldt / Roe wave-speed bounds in the
textbook form (Roe-averaged H and transverse velocities, Toro's star state).
The stage kernel evaluates an algebraically equal arrangement with fewer FP64
operations (its adjoint the same one, with u~ = w_L u_L + w_R u_R):
- one reciprocal square root q = 1/sqrt(rho_L rho_R) gives 1/rho_L = rho_R q^2,
  1/rho_R = rho_L q^2 and the Roe ratio r = sqrt(rho_R/rho_L) = rho_R q;
- Roe weights w_L = 1/(1 + r), w_R = r w_L, and u~ = u_L - w_R (u_L - u_R);
- the Roe sound speed as w_L c_L^2 + w_R c_R^2 + (gamma-1)/2 w_L w_R |u_L - u_R|^2,
  equal to (gamma-1)(H~ - |u~|^2/2) because H_K = c_K^2/(gamma-1) + |u_K|^2/2 and
  w_L + w_R = 1;
- inside the fan t = u_K + g = S* (S_K - u_K)/(S_K - S*), and
  F0 = rho_K t, F1 = F0 u_K + p_K + g m_K, F2 = v_K F0, F3 = w_K F0,
  F4 = h_K t + g m_K S* with g = t - u_K and m_K = rho_K (S_K - u_K).

This file writes that arrangement out in plain Python (double precision) and
checks it against the oracle's flux and fan speeds on random subsonic and
supersonic states: a check of the algebra behind the GPU's reading, in
rounding-level agreement.  It runs on the CPU only.
"""
import math

import numpy as np

from oracle import oracle as orc

G = 1.4


def arranged_hllc(WL, WR, gamma=G):
    """(F, S_L, S_R, S*) in the CUDA path's arrangement (exact sqrt / division)."""
    rL, uL, vL, wL, pL = (float(x) for x in WL)
    rR, uR, vR, wR, pR = (float(x) for x in WR)
    q = 1.0 / math.sqrt(rL * rR)
    q2 = q * q
    iL, iR = rR * q2, rL * q2
    cL2, cR2 = gamma * pL * iL, gamma * pR * iR
    cL, cR = math.sqrt(cL2), math.sqrt(cR2)
    r = rR * q
    wl = 1.0 / (1.0 + r)
    wr = r * wl
    ut = uL - wr * (uL - uR)
    du2 = (uL - uR) ** 2 + (vL - vR) ** 2 + (wL - wR) ** 2
    ct = math.sqrt(0.5 * (gamma - 1.0) * wl * wr * du2 + wl * cL2 + wr * cR2)
    SL = min(uL - cL, ut - ct)
    SR = max(uR + cR, ut + ct)
    dL, dR = SL - uL, SR - uR
    mL, mR = rL * dL, rR * dR
    Ss = (pR - pL + mL * uL - mR * uR) / (mL - mR)
    left = Ss >= 0.0
    rK, uK, vK, wK, pK = (rL, uL, vL, wL, pL) if left else (rR, uR, vR, wR, pR)
    SK, mK, dK = (SL, mL, dL) if left else (SR, mR, dR)
    fan = SL < 0.0 if left else SR > 0.0
    t = Ss * dK / (SK - Ss) if fan else uK
    g = t - uK
    hK = 0.5 * rK * (uK * uK + vK * vK + wK * wK) + gamma / (gamma - 1.0) * pK
    F0 = rK * t
    F = np.array([F0, F0 * uK + pK + g * mK, vK * F0, wK * F0, hK * t + g * mK * Ss])
    return F, SL, SR, Ss


def states(n, seed, mach):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = rng.uniform(0.05, 5.0)
        p = rng.uniform(1e-3, 5.0)
        c = math.sqrt(G * p / r)
        vel = rng.uniform(-mach, mach, 3) * c
        out.append(np.array([r, *vel, p]))
    return out


def check(WL, WR, tol):
    F_ref, d = orc.hllc(WL, WR, detail=True)
    F, SL, SR, Ss = arranged_hllc(WL, WR)
    scale = max(float(np.max(np.abs(F_ref))), 1e-300)
    assert float(np.max(np.abs(F - F_ref))) <= tol * scale
    speed = max(abs(d["SL"]), abs(d["SR"]), 1e-300)
    assert abs(SL - d["SL"]) <= tol * speed and abs(SR - d["SR"]) <= tol * speed
    assert abs(Ss - d["Ss"]) <= tol * speed


def test_arrangement_matches_oracle_subsonic():
    for a, b in zip(states(2000, 1, 0.8), states(2000, 2, 0.8)):
        check(a, b, 1e-13)


def test_arrangement_matches_oracle_supersonic_and_strong_jumps():
    # Mach up to 10 and density / pressure jumps of up to ~10^3 across the face
    for a, b in zip(states(2000, 3, 10.0), states(2000, 4, 10.0)):
        check(a, b, 1e-12)


def test_arrangement_sod_face_and_mirror():
    sod_l = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    sod_r = np.array([0.125, 0.0, 0.0, 0.0, 0.1])
    check(sod_l, sod_r, 1e-14)
    a = np.array([1.3, 0.4, -0.2, 0.1, 0.9])
    b = np.array([0.7, -0.3, 0.5, 0.0, 1.4])
    F, *_ = arranged_hllc(a, b)
    mir = lambda W: np.array([W[0], -W[1], W[2], W[3], W[4]])
    Fm, *_ = arranged_hllc(mir(b), mir(a))
    # mirror: F(mir R, mir L) = -mir(F(L, R)) for the mass, normal-momentum-flipped components
    assert np.max(np.abs(Fm - np.array([-F[0], F[1], -F[2], -F[3], -F[4]]))) <= 1e-13 * np.max(np.abs(F))


def test_roe_sound_speed_identity_where_the_textbook_form_cancels():
    """At high relative Mach number (gamma-1)(H~ - |u~|^2/2) is a small
    difference of large numbers; the arranged form is a sum of non-negative
    terms.  Both agree to the rounding of the textbook form."""
    rng = np.random.default_rng(9)
    for _ in range(500):
        rL, rR = rng.uniform(0.1, 10.0, 2)
        pL, pR = rng.uniform(1e-4, 1.0, 2)
        uL, uR = rng.uniform(-50.0, 50.0, 2)
        wl = math.sqrt(rL) / (math.sqrt(rL) + math.sqrt(rR))
        wr = 1.0 - wl
        HL = G / (G - 1) * pL / rL + 0.5 * uL * uL
        HR = G / (G - 1) * pR / rR + 0.5 * uR * uR
        ut = wl * uL + wr * uR
        textbook = (G - 1) * (wl * HL + wr * HR - 0.5 * ut * ut)
        arranged = wl * G * pL / rL + wr * G * pR / rR + 0.5 * (G - 1) * wl * wr * (uL - uR) ** 2
        big = (G - 1) * max(wl * HL + wr * HR, 0.5 * ut * ut)
        assert arranged > 0.0
        assert abs(arranged - textbook) <= 64 * np.finfo(float).eps * big
