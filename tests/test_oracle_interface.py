"""Pins of the interface constitutive oracle (oracle/interface.py; Sec. 2.2 and the
elastic predictor - plastic corrector of Sec. 3.1.1) against what the mechanics fixes:

* inside the yield surfaces the step is elastic: T' = T'^n + C dd and C^ep = C;
* perfect Coulomb plasticity (no softening) has a closed-form multiplier and tangent,
  written out here from the radial return: dl = F_trial / (K_s + f psi K_n) and
  C^ep = C - (terms of the return), including the rotation of the shear direction;
* a perfect tensile cut-off holds T'_n = sigma_p and has C^ep = diag(K_s, K_s, 0);
* after any return the active yield function vanishes (at the cone's apex: no shear
  traction and f T'_n = c), the inelastic increment points
  along the flow direction, the elastic law T' - T'^n = C (dd - d delta^p) holds and the
  internal variables are the maxima the paper defines;
* the complex-step tangent equals central finite differences of the update;
* in the rigid limit a monotonic shear under a fixed normal traction follows the linear
  slip-weakening law tau = f(delta_s) sigma_n, and a monotonic opening follows the linear
  cohesive law T'_n = sigma_p (1 - delta_n / w_c) down to the open state;
* an open pre-existing fracture carries no traction and re-enters contact exactly when
  its normal inelastic DD would pass below the residual width.
"""
import math

import numpy as np
import pytest

from oracle import interface as I


def params(**kw):
    base = dict(Ks=10.0, Kn=20.0, fp=0.6, fr=0.3, psip=0.1, dc=0.2, cp=0.1, sigp=0.5, wc=0.4, alphaR=0.5)
    base.update(kw)
    return I.Params(**base)


def test_elastic_inside_the_yield_surfaces():
    P = params()
    T = np.array([0.2, -0.1, -1.0])
    dd = np.array([0.01, 0.02, -0.01])
    T1, dp1, chi1, mode, C = I.step(P, T, np.zeros(3), np.zeros(3), dd)
    assert mode == I.ELASTIC
    assert np.allclose(T1, T + np.array([P.Ks, P.Ks, P.Kn]) * dd, rtol=0, atol=1e-15)
    assert np.array_equal(dp1, np.zeros(3)) and np.array_equal(chi1, np.zeros(3))
    assert np.allclose(C, np.diag([P.Ks, P.Ks, P.Kn]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_perfect_coulomb_closed_form(seed):
    rng = np.random.default_rng(seed)
    f, psi, c = rng.uniform(0.3, 0.8), rng.uniform(0.0, 0.3), rng.uniform(0.0, 0.2)
    Ks, Kn = rng.uniform(5, 20), rng.uniform(5, 40)
    # no softening: slip and damage scales far beyond the step
    P = I.Params(Ks=Ks, Kn=Kn, fp=f, fr=f, psip=psi, dc=1e300, cp=c, sigp=10.0, wc=1e300, alphaR=0.0)
    T = np.array([rng.normal() * 0.1, rng.normal() * 0.1, -rng.uniform(0.5, 2.0)])
    dd = np.array([rng.normal(), rng.normal(), rng.normal() * 0.01]) * 0.3
    Ttr = T + np.array([Ks, Ks, Kn]) * dd
    tau = math.hypot(Ttr[0], Ttr[1])
    F = tau + f * Ttr[2] - c
    assert F > 0.0
    s = Ttr[:2] / tau
    den = Ks + f * psi * Kn
    dl = F / den
    ref_T = np.array([(tau - Ks * dl) * s[0], (tau - Ks * dl) * s[1], Ttr[2] - Kn * psi * dl])
    # tangent: d(dl) = (K_s s . d dd_s + f K_n d dd_n) / den; d s = K_s (I - s s^T) d dd_s / tau
    a = np.array([Ks * s[0], Ks * s[1], f * Kn]) / den
    Cref = np.zeros((3, 3))
    P2 = np.eye(2) - np.outer(s, s)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1.0
        dtau = Ks * s @ e[:2]
        dds = Ks * P2 @ e[:2] / tau
        ddl = a[j]
        Cref[:2, j] = (dtau - Ks * ddl) * s + (tau - Ks * dl) * dds
        Cref[2, j] = Kn * e[2] - Kn * psi * ddl
    T1, dp1, chi1, mode, C = I.step(P, T, np.zeros(3), np.zeros(3), dd)
    assert mode == I.COULOMB
    assert np.abs(T1 - ref_T).max() <= 1e-12 * np.abs(ref_T).max()
    assert np.abs(dp1 - dl * np.array([s[0], s[1], psi])).max() <= 1e-12 * dl
    assert np.abs(C - Cref).max() <= 1e-9 * np.abs(Cref).max()


def test_perfect_tensile_cutoff():
    P = params(sigp=0.5, wc=1e300, cp=0.2, fp=0.6, fr=0.6)
    T = np.array([0.05, 0.0, 0.0])
    dd = np.array([0.0, 0.01, 0.1])                 # pure opening: T_n,trial = 2 > sigma_p
    T1, dp1, chi1, mode, C = I.step(P, T, np.zeros(3), np.zeros(3), dd)
    assert mode == I.TENSILE
    Ttr = T + np.array([P.Ks, P.Ks, P.Kn]) * dd
    assert np.allclose(T1, [Ttr[0], Ttr[1], 0.5], rtol=0, atol=1e-14)
    assert np.allclose(dp1, [0, 0, (Ttr[2] - 0.5) / P.Kn], rtol=0, atol=1e-15)
    assert np.allclose(C, np.diag([P.Ks, P.Ks, 0.0]), rtol=0, atol=1e-9)


def random_yielding_state(rng, P):
    T = np.array([rng.normal() * 0.2, rng.normal() * 0.2, -rng.uniform(0.2, 1.5)])
    dp = np.array([rng.normal() * 0.02, rng.normal() * 0.02, abs(rng.normal()) * 0.005])
    chis = math.hypot(dp[0], dp[1]) * rng.uniform(1.0, 1.5)
    chit = float(np.linalg.norm(dp)) * rng.uniform(1.0, 1.5)
    chi = np.array([chis, chit, abs(rng.normal()) * 0.002])
    dd = np.array([rng.normal(), rng.normal(), rng.normal() * 0.3]) * 0.08
    return T, dp, chi, dd


def yield_values(P, T1, chi1):
    tau = math.hypot(T1[0], T1[1])
    return (tau + I.friction(P, chi1[0]) * T1[2] - I.cohesion(P, chi1[1]),
            T1[2] - I.tensile_strength(P, chi1[1]))


@pytest.mark.parametrize("seed", range(40))
def test_return_lies_on_the_yield_surface_with_the_flow_rule(seed):
    rng = np.random.default_rng(100 + seed)
    P = params(Ks=rng.uniform(8, 20), Kn=rng.uniform(10, 40))
    T, dp, chi, dd = random_yielding_state(rng, P)
    T1, dp1, chi1, mode, C = I.step(P, T, dp, chi, dd)
    K = np.array([P.Ks, P.Ks, P.Kn])
    ddp = dp1 - dp
    if mode != I.OPEN:
        # elastic law on the elastic part of the increment
        assert np.abs(T1 - (T + K * (dd - ddp))).max() <= 1e-12 * (1 + np.abs(T1).max())
    Fc, Ft = yield_values(P, T1, chi1)
    if mode == I.COULOMB:
        assert abs(Fc) <= 1e-12 and Ft <= 1e-12
        Ttr = T + K * dd
        s = Ttr[:2] / math.hypot(Ttr[0], Ttr[1])
        dl = math.hypot(ddp[0], ddp[1])
        psi1 = I.dilatancy(P, chi1[0])
        assert np.abs(ddp - dl * np.array([s[0], s[1], psi1])).max() <= 1e-12 * max(dl, 1e-300)
        assert np.abs(T1[:2] / math.hypot(T1[0], T1[1]) - s).max() <= 1e-12
        assert abs(chi1[2] - (chi[2] + psi1 * dl)) <= 1e-15
    elif mode == I.TENSILE:
        assert abs(Ft) <= 1e-12 and Fc <= 1e-12
        assert ddp[0] == 0.0 and ddp[1] == 0.0 and ddp[2] >= 0.0
    elif mode == I.APEX:
        assert T1[0] == 0.0 and T1[1] == 0.0 and abs(Fc) <= 1e-12
        Ttr = T + K * dd
        assert np.abs(ddp[:2] - Ttr[:2] / P.Ks).max() <= 1e-15
    elif mode == I.ELASTIC:
        assert Fc <= 0.0 and Ft <= 0.0
    assert chi1[0] == pytest.approx(max(chi[0], math.hypot(dp1[0], dp1[1])), rel=1e-15, abs=0)
    assert chi1[1] == pytest.approx(max(chi[1], float(np.linalg.norm(dp1))), rel=1e-15, abs=0)


def test_modes_are_all_reached():
    seen = set()
    for seed in range(40):
        rng = np.random.default_rng(100 + seed)
        P = params(Ks=rng.uniform(8, 20), Kn=rng.uniform(10, 40))
        T, dp, chi, dd = random_yielding_state(rng, P)
        seen.add(I.step(P, T, dp, chi, dd)[3])
    assert {I.ELASTIC, I.COULOMB} <= seen
    P = params()
    assert I.step(P, np.zeros(3), np.zeros(3), np.zeros(3), np.array([0, 0, 0.1]))[3] == I.TENSILE
    assert I.step(P, np.zeros(3), np.zeros(3), np.array([0, 0.5, 0]), np.array([0, 0, 0.1]))[3] == I.OPEN


@pytest.mark.parametrize("seed", range(12))
def test_tangent_matches_central_differences(seed):
    rng = np.random.default_rng(300 + seed)
    P = params(Ks=rng.uniform(8, 20), Kn=rng.uniform(10, 40))
    T, dp, chi, dd = random_yielding_state(rng, P)
    if seed % 3 == 2:                                  # a tensile return
        T = np.array([0.02, -0.01, 0.1])
        dd = np.array([0.001, 0.0, 0.05])
        dp, chi = np.zeros(3), np.zeros(3)
    T1, _, _, mode, C = I.step(P, T, dp, chi, dd)
    h = 1e-7
    Cfd = np.empty((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        Tp = I.step(P, T, dp, chi, dd + e)[0]
        Tm = I.step(P, T, dp, chi, dd - e)[0]
        assert I.step(P, T, dp, chi, dd + e)[3] == mode
        Cfd[:, j] = (Tp - Tm) / (2 * h)
    assert np.abs(C - Cfd).max() <= 1e-6 * max(P.Ks, P.Kn), (mode, C, Cfd)


def test_rigid_limit_follows_linear_slip_weakening():
    sig_n = 2.0
    P = I.Params(Ks=1e7, Kn=1e7, fp=0.6, fr=0.3, psip=0.0, dc=0.1, cp=0.0, sigp=0.0, wc=0.0, alphaR=0.0)
    # fully damaged pre-existing fault (w_c = 0): no cohesion, contact under sigma_n
    T = np.array([0.0, 0.0, -sig_n])
    dp = np.zeros(3)
    chi = np.zeros(3)
    for k in range(30):
        T, dp, chi, mode, _ = I.step(P, T, dp, chi, np.array([0.01, 0.0, 0.0]))
        if mode == I.COULOMB:
            slip = dp[0]
            f = 0.3 + 0.3 * max(0.0, 1.0 - slip / 0.1)
            assert T[0] == pytest.approx(f * sig_n, rel=1e-9)  # K_s dl resolves to 1e7 ulp(dl)
    assert dp[0] > 0.25 and T[0] == pytest.approx(0.3 * sig_n, rel=1e-9)


def test_rigid_limit_follows_linear_cohesive_law():
    P = I.Params(Ks=1e7, Kn=1e7, fp=0.6, fr=0.6, psip=0.0, dc=1.0, cp=0.0, sigp=1.0, wc=0.2, alphaR=0.5)
    T, dp, chi = np.zeros(3), np.zeros(3), np.zeros(3)
    modes = []
    for k in range(30):
        T, dp, chi, mode, C = I.step(P, T, dp, chi, np.array([0.0, 0.0, 0.01]))
        modes.append(mode)
        if mode == I.TENSILE:
            assert T[2] == pytest.approx(1.0 - dp[2] / 0.2, rel=1e-9)  # K_n dl resolves to 1e7 ulp(dl)
            S = 1.0 / 0.2                       # softening rate sigma_p / w_c
            assert C[2, 2] == pytest.approx(-S / (1.0 - S / P.Kn), rel=1e-9)
        if mode == I.OPEN:
            assert np.array_equal(T, np.zeros(3)) and np.abs(C).max() == 0.0
    assert modes[0] == I.TENSILE and modes[-1] == I.OPEN and I.COULOMB not in modes


def test_open_fracture_and_contact():
    Kn, s0 = 20.0, 1.0
    P = params(Kn=Kn, sigp=0.0, wc=0.0, cp=0.0, alphaR=0.0)   # pre-existing fracture
    T = np.array([0.0, 0.0, -s0])
    T1, dp1, chi1, mode, C = I.step(P, T, np.zeros(3), np.zeros(3), np.array([0.0, 0.0, 2 * s0 / Kn]))
    assert mode == I.OPEN and np.array_equal(T1, np.zeros(3)) and np.abs(C).max() == 0.0
    assert dp1[2] == pytest.approx(s0 / Kn, rel=1e-15)
    # closing by less than the gap stays open ...
    T2, dp2, chi2, mode2, _ = I.step(P, T1, dp1, chi1, np.array([0.0, 0.0, -0.5 * s0 / Kn]))
    assert mode2 == I.OPEN and dp2[2] == pytest.approx(0.5 * s0 / Kn, rel=1e-12)
    # ... closing past it comes back into contact with delta^p_n at the residual width 0
    T3, dp3, chi3, mode3, C3 = I.step(P, T2, dp2, chi2, np.array([0.0, 0.0, -1.0 * s0 / Kn]))
    assert mode3 == I.ELASTIC and dp3[2] == 0.0
    assert T3[2] == pytest.approx(-0.5 * s0, rel=1e-12)
    assert np.allclose(C3, np.diag([P.Ks, P.Ks, Kn]), rtol=0, atol=1e-9)


def test_mode_selection_function():
    P = params(cp=0.5, sigp=0.5, wc=1e300, fp=0.6, fr=0.6, psip=0.0)
    zero = np.zeros(3)
    # deep compression with shear beyond friction: Coulomb
    assert I.step(P, np.array([2.0, 0, -1.0]), zero, zero, zero)[3] == I.COULOMB
    # tension beyond the cut-off with little shear: tensile
    assert I.step(P, np.array([0.01, 0, 1.0]), zero, zero, zero)[3] == I.TENSILE
    # both violated near the corner (T'_n = 0.5, tau = 0.2): the sign of h decides
    f = 0.6
    a = math.sqrt(1 + f * f) - f
    for Tn, tau in [(0.6, 0.3), (0.55, 0.4), (0.7, 0.1), (0.8, 0.25)]:
        assert tau + f * Tn - 0.5 > 0 and Tn - 0.5 > 0
        h = tau - (0.5 - f * 0.5) - a * (Tn - 0.5)
        mode = I.step(P, np.array([tau, 0, Tn]), zero, zero, zero)[3]
        assert mode == (I.COULOMB if h > 0 else I.TENSILE), (Tn, tau, h, mode)


def test_apex_return():
    # the cone's apex c/f = 1/6 lies below the cut-off 0.5: a tensile trial with shear
    # returns to the apex
    P = params(cp=0.1, sigp=0.5, wc=1e300, fp=0.6, fr=0.6, dc=1e300)
    zero = np.zeros(3)
    T1, dp1, chi1, mode, C = I.step(P, np.array([0.2, 0.1, 0.4]), zero, zero, zero)
    assert mode == I.APEX
    assert T1[0] == 0.0 and T1[1] == 0.0 and T1[2] == pytest.approx(0.1 / 0.6, rel=1e-14)
    assert np.allclose(dp1, [0.2 / P.Ks, 0.1 / P.Ks, (0.4 - 0.1 / 0.6) / P.Kn], rtol=1e-14, atol=0)
    assert np.abs(C).max() <= 1e-9                     # perfect apex: no stiffness left
