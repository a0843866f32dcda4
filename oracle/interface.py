"""FP64 CPU oracle of the interface constitutive update and its consistent tangent
(Sec. 2.2: the poroelastoplastic interface law, its yield criteria, flow rules and
damage; Sec. 3.1.1: the elastic predictor - plastic corrector integration and the
consistent tangent C^ep = d(Delta T')/d(Delta delta) of eq. jac_mech).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path; it shares no
code with the CUDA library.

Per collocation point, in the element's local frame (s1, s2, n), one time step takes the
state at t^n -- effective traction T', inelastic DD delta^p, internal variables chi_s
(largest inelastic slip magnitude) and chi_t (largest inelastic DD magnitude), and the
dilatant part w_dil of the residual width -- and an increment Delta delta of the total
DD, and returns the state at t^(n+1), the active mode and C^ep.  The law (Sec. 2.2):

    T' - T'^n = C (Delta delta - Delta delta^p),   C = diag(K_s, K_s, K_n)
    Coulomb   F_c = |tau| + f(chi_s) T'_n - c(chi_t),   flow  d delta^p = dl (s_hat + psi(chi_s) n)
    tension   F_t = T'_n - sigma_t(chi_t),              flow  d delta^p = dl n
    f = (f_p - f_r) W(chi_s / d_c) + f_r,  psi = psi_p W(chi_s / d_c),
    c = c_p W(chi_t / w_c),  sigma_t = sigma_p W(chi_t / w_c),  W(x) = max(0, 1 - x)

Readings taken where the paper is silent or leaves the details to its supplement:
  R1 backward Euler: f, psi, c, sigma_t and the internal variables are those of
     t^(n+1); chi_s^(n+1) = max(chi_s^n, |delta^p_s^(n+1)|), chi_t^(n+1) =
     max(chi_t^n, |delta^p^(n+1)|) (the paper's maxima over time of the magnitudes);
  R2 cohesion and tensile strength soften with chi_t (the paper's C(chi_n) and
     sigma_t(chi_n) name the variable it defines as chi_t);
  R3 the failure mode is chosen once, at the trial state with the strengths of t^n, by
     the sign of h = |tau| - (c - f sigma_t) - a (T'_n - sigma_t), a = sqrt(1 + f^2) - f:
     h > 0 Coulomb, otherwise tension;
  R3a the apex: where the Coulomb return has no root before the shear traction vanishes
     (the cone's apex c/f lies below the tensile cut-off), the step returns to the apex:
     all of the trial shear is inelastic (tau = 0) and the normal inelastic increment mu
     solves f(chi_s) (T'_n,trial - K_n mu) = c(chi_t) on [0, T'_n,trial / K_n], w_dil
     unchanged; an apex return that reaches chi_t >= w_c ends in the open state;
  R4 the Coulomb return keeps the trial shear direction (C is isotropic in the shear
     plane), so it is a scalar equation g(dl) = 0 for the plastic multiplier on
     [0, |tau_trial| / K_s];
  R5 damage: the interface is fully damaged when w_c = 0 (a pre-existing fracture,
     sigma_p = 0) or chi_t >= w_c.  A fully damaged interface in tension is open:
     T' = 0 (both stiffnesses vanish), all of Delta delta + C^-1 T'^n is inelastic and
     C^ep = 0.  A tensile return that reaches chi_t >= w_c ends in that open state;
  R6 contact of a fully damaged interface (the Signorini condition): the residual width
     is w_R = alpha_R w_c + w_dil; the closed state keeps its normal inelastic DD at
     min(delta^p_n, w_R); the interface is open when the trial normal traction of that
     closed state is tensile, otherwise it is in contact and frictional (c = 0);
  R7 w_dil grows by the dilatant opening psi dl of every Coulomb return (the paper's
     evolution of w_R by shear-induced dilation);
  R8 constant K_n and K_s (the constant-stiffness option of the paper);
  R9 unique local return: the multiplier equation is taken to have a single root on its
     bracket (interface stiffness above the softening rate of the strengths); the root
     is found by bisection;
  R10 C^ep is the derivative of T'^(n+1) with respect to Delta delta within the active
     mode, computed by complex-step differentiation (Squire and Trapp, 1998; Martins,
     Sturdza and Alonso, 2003): every quantity is carried as a complex number, branch
     decisions use real parts, and the multiplier's imaginary part is driven to the
     complex root of its equation by a fixed-slope iteration.

Plain Python over complex scalars, one point at a time: for the small cases of the tests.
"""
from __future__ import annotations

import cmath
from dataclasses import dataclass

import numpy as np

ELASTIC, COULOMB, TENSILE, OPEN, APEX = 0, 1, 2, 3, 4


@dataclass
class Params:
    Ks: float        # shear stiffness of the interface
    Kn: float        # normal stiffness
    fp: float        # peak friction coefficient
    fr: float        # residual friction coefficient
    psip: float      # peak dilatancy coefficient
    dc: float        # slip-weakening distance (> 0)
    cp: float        # peak cohesion
    sigp: float      # peak tensile strength
    wc: float        # critical inelastic DD of cohesion and tensile strength (0: pre-existing fracture)
    alphaR: float    # residual width after full damage, as a fraction of w_c

    def as_array(self):
        return np.array([self.Ks, self.Kn, self.fp, self.fr, self.psip, self.dc, self.cp, self.sigp,
                         self.wc, self.alphaR], dtype=np.float64)


def _cmax(a, b):
    return a if a.real >= b.real else b


def _soft(scale, chi):
    """W(chi / scale) with W(x) = max(0, 1 - x); a zero scale is fully softened."""
    if scale <= 0.0:
        return 0.0
    x = chi / scale
    return 0.0 if x.real >= 1.0 else 1.0 - x


def friction(P, chis):
    return (P.fp - P.fr) * _soft(P.dc, chis) + P.fr


def dilatancy(P, chis):
    return P.psip * _soft(P.dc, chis)


def cohesion(P, chit):
    return P.cp * _soft(P.wc, chit)


def tensile_strength(P, chit):
    return P.sigp * _soft(P.wc, chit)


def _norm(*v):
    return cmath.sqrt(sum(x * x for x in v))


def _root(g, hi):
    """Root of g on [0, hi] (g(0) > 0 >= g(hi) in real part) by bisection on the real
    part, then its complex continuation by a fixed-slope iteration (reading R10).  No
    return (0) when g(0) <= 0."""
    if g(0.0).real <= 0.0:
        return 0.0
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if g(mid).real > 0.0:
            lo = mid
        else:
            hi = mid
    x = 0.5 * (lo + hi)
    h = 1e-7 * max(x, 1e-300)
    slope = (g(x + h).real - g(x - h).real) / (2.0 * h) if x > h else (g(x + h).real - g(x).real) / h
    if slope == 0.0:
        return x
    z = complex(x)
    for _ in range(8):
        z = z - g(z) / slope
    return z


def _open(P, T, dp, dd, chis, chit):
    dp1 = [dp[0] + dd[0] + T[0] / P.Ks, dp[1] + dd[1] + T[1] / P.Ks, dp[2] + dd[2] + T[2] / P.Kn]
    return dict(T=[0.0 * dd[0], 0.0 * dd[0], 0.0 * dd[0]], dp=dp1,
                chis=_cmax(complex(chis), _norm(dp1[0], dp1[1])), chit=_cmax(complex(chit), _norm(*dp1)),
                mode=OPEN)


def _apex(P, Ttr, dp, chis, chit, wdil):
    """Return to the apex of the Coulomb cone (reading R3a)."""
    tau_tr = _norm(Ttr[0], Ttr[1])
    if tau_tr.real > 0.0:
        dps = [dp[0] + Ttr[0] / P.Ks, dp[1] + Ttr[1] / P.Ks]
    else:
        dps = [complex(dp[0]), complex(dp[1])]
    chis1 = _cmax(complex(chis), _norm(*dps))
    f1 = friction(P, chis1)

    def chit_of(mu):
        return _cmax(complex(chit), _norm(dps[0], dps[1], dp[2] + mu))

    def g(mu):
        return f1 * (Ttr[2] - P.Kn * mu) - cohesion(P, chit_of(mu))

    mu = _root(g, Ttr[2].real / P.Kn)
    return dict(T=[0.0 * Ttr[0], 0.0 * Ttr[0], Ttr[2] - P.Kn * mu], dp=[dps[0], dps[1], dp[2] + mu],
                chis=chis1, chit=chit_of(mu), wdil=complex(wdil), mode=APEX)


def _coulomb(P, Ttr, dp, chis, chit, wdil):
    """Return on F_c = 0 with the non-associated flow (readings R1, R4), or to the apex."""
    tau_tr = _norm(Ttr[0], Ttr[1])
    if tau_tr.real <= 0.0:
        return _apex(P, Ttr, dp, chis, chit, wdil)
    s = (Ttr[0] / tau_tr, Ttr[1] / tau_tr)

    def state(dl):
        chis1 = _cmax(complex(chis), _norm(dp[0] + dl * s[0], dp[1] + dl * s[1]))
        psi1 = dilatancy(P, chis1)
        dp1 = [dp[0] + dl * s[0], dp[1] + dl * s[1], dp[2] + dl * psi1]
        chit1 = _cmax(complex(chit), _norm(*dp1))
        return chis1, chit1, psi1, dp1, tau_tr - P.Ks * dl, Ttr[2] - P.Kn * psi1 * dl

    def g(dl):
        chis1, chit1, psi1, dp1, tau1, Tn1 = state(dl)
        return tau1 + friction(P, chis1) * Tn1 - cohesion(P, chit1)

    hi = tau_tr.real / P.Ks
    if g(hi).real > 0.0:
        return _apex(P, Ttr, dp, chis, chit, wdil)
    dl = _root(g, hi)
    chis1, chit1, psi1, dp1, tau1, Tn1 = state(dl)
    return dict(T=[tau1 * s[0], tau1 * s[1], Tn1], dp=dp1, chis=chis1, chit=chit1, wdil=wdil + psi1 * dl,
                mode=COULOMB)


def _tensile(P, Ttr, dp, chis, chit):
    """Return on F_t = 0 with the associated flow along n."""
    def chit_of(dl):
        return _cmax(complex(chit), _norm(dp[0], dp[1], dp[2] + dl))

    def g(dl):
        return Ttr[2] - P.Kn * dl - tensile_strength(P, chit_of(dl))

    dl = _root(g, Ttr[2].real / P.Kn)
    return dict(T=[Ttr[0], Ttr[1], Ttr[2] - P.Kn * dl], dp=[dp[0], dp[1], dp[2] + dl],
                chis=complex(chis), chit=chit_of(dl), mode=TENSILE)


def fully_damaged(P, chit):
    return P.wc <= 0.0 or chit >= P.wc


def update(P, T, dp, chi, dd):
    """One constitutive step.  T, dp: length-3 real (s1, s2, n); chi = (chi_s, chi_t,
    w_dil); dd: the DD increment (complex entries allowed, reading R10).  Returns a dict
    with T, dp (lists), chis, chit, wdil and mode."""
    chis, chit, wdil = float(chi[0]), float(chi[1]), float(chi[2])
    dd = [complex(x) for x in dd]
    T = [float(x) for x in T]
    dp = [float(x) for x in dp]
    if fully_damaged(P, chit):                                  # reading R6
        wR = P.alphaR * P.wc + wdil
        dpn_c = min(dp[2], wR)
        Ttr = [T[0] + P.Ks * dd[0], T[1] + P.Ks * dd[1], T[2] + P.Kn * (dd[2] - (dpn_c - dp[2]))]
        if Ttr[2].real > 0.0:
            out = _open(P, T, dp, dd, chis, chit)
            out["wdil"] = complex(wdil)
            return out
        dpc = [dp[0], dp[1], dpn_c]
        Fc = _norm(Ttr[0], Ttr[1]) + friction(P, chis) * Ttr[2]
        if Fc.real <= 0.0:
            return dict(T=Ttr, dp=[complex(x) for x in dpc], chis=complex(chis), chit=complex(chit),
                        wdil=complex(wdil), mode=ELASTIC)
        return _coulomb(P, Ttr, dpc, chis, chit, wdil)
    Ttr = [T[0] + P.Ks * dd[0], T[1] + P.Ks * dd[1], T[2] + P.Kn * dd[2]]
    tau_tr = _norm(Ttr[0], Ttr[1])
    f0, c0, st0 = friction(P, chis), cohesion(P, chit), tensile_strength(P, chit)
    Fc = tau_tr + f0 * Ttr[2] - c0
    Ft = Ttr[2] - st0
    if Fc.real <= 0.0 and Ft.real <= 0.0:
        return dict(T=Ttr, dp=[complex(x) for x in dp], chis=complex(chis), chit=complex(chit),
                    wdil=complex(wdil), mode=ELASTIC)
    a = np.sqrt(1.0 + f0 * f0) - f0
    h = tau_tr.real - (c0 - f0 * st0) - a * (Ttr[2].real - st0)  # reading R3
    if h > 0.0:
        out = _coulomb(P, Ttr, dp, chis, chit, wdil)
    else:
        out = _tensile(P, Ttr, dp, chis, chit)
        out["wdil"] = complex(wdil)
    if out["mode"] != COULOMB and fully_damaged(P, out["chit"].real):   # readings R3a, R5
        out = _open(P, T, dp, dd, chis, chit)
        out["wdil"] = complex(wdil)
    return out


def tangent(P, T, dp, chi, dd, h=1e-30):
    """C^ep = d T'^(n+1) / d Delta delta (3x3, row = traction component) by complex step."""
    C = np.empty((3, 3))
    for j in range(3):
        z = [complex(x) for x in dd]
        z[j] += 1j * h
        out = update(P, T, dp, chi, z)
        for i in range(3):
            C[i, j] = complex(out["T"][i]).imag / h
    return C


def step(P, T, dp, chi, dd):
    """Real outputs of one step: (T1[3], dp1[3], chi1[3], mode, Cep[3x3])."""
    out = update(P, T, dp, chi, dd)
    T1 = np.array([complex(x).real for x in out["T"]])
    dp1 = np.array([complex(x).real for x in out["dp"]])
    chi1 = np.array([complex(out["chis"]).real, complex(out["chit"]).real, complex(out["wdil"]).real])
    return T1, dp1, chi1, out["mode"], tangent(P, T, dp, chi, dd)


def step_all(P, T, dp, chi, dd):
    """step() over arrays of points: T, dp, chi, dd of shape (n, 3)."""
    n = T.shape[0]
    T1 = np.empty((n, 3))
    dp1 = np.empty((n, 3))
    chi1 = np.empty((n, 3))
    mode = np.empty(n, dtype=np.int32)
    cep = np.empty((n, 3, 3))
    for e in range(n):
        T1[e], dp1[e], chi1[e], mode[e], cep[e] = step(P, T[e], dp[e], chi[e], dd[e])
    return T1, dp1, chi1, mode, cep
