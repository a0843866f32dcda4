// Interface constitutive update (Sec. 2.2: the poroelastoplastic interface law with a
// Coulomb yield surface, a tensile cut-off, softening of friction, dilatancy, cohesion
// and tensile strength, damage, opening and contact) integrated by an elastic predictor
// and plastic corrector (Sec. 3.1.1), with the consistent tangent
// C^ep = d(Delta T') / d(Delta delta) of eq. jac_mech.  One thread per collocation point,
// FP64.
//
// The tangent is exact: the return is evaluated in forward-mode dual numbers.  The
// plastic multiplier is found in plain arithmetic (Newton safeguarded by bisection, the
// slope from a one-component dual), and one more Newton step in four-component duals
// (three for Delta delta, one for the multiplier) gives its derivative by the implicit
// function theorem: d(dl) = -(dg/d dd) / (dg/d dl) at the root.  The rest of the return
// is then re-evaluated in three-component duals, whose derivative parts are C^ep.
//
// Branches (the active mode, the maxima of the internal variables) are taken on values,
// so C^ep is the derivative within the active mode.  Two passes: one classifies every
// point and finishes the elastic and open ones, then each kind of return (Coulomb,
// tensile, apex) runs over its own list, so that a warp follows one branch.  The choices the paper leaves open
// are those stated with hm_interface_update in hmat.h.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace hm {
namespace {

enum : int32_t { M_ELASTIC = 0, M_COULOMB = 1, M_TENSILE = 2, M_OPEN = 3, M_APEX = 4 };
constexpr int N_MODES = 5;
constexpr int ST_NOROOT = 1;  // a multiplier bracket without a sign change or no convergence

struct Prm {
    double Ks, Kn, fp, fr, psip, dc, cp, sigp, wc, alphaR;
};

// ---------------------------------------------------------------- dual numbers
template <int K>
struct Dual {
    double v;
    double d[K];
};

template <int K>
__device__ __forceinline__ Dual<K> cst(double x) {
    Dual<K> r;
    r.v = x;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = 0.0;
    return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(Dual<K> a, Dual<K> b) {
    a.v += b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) a.d[i] += b.d[i];
    return a;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(Dual<K> a, Dual<K> b) {
    a.v -= b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) a.d[i] -= b.d[i];
    return a;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(Dual<K> a, Dual<K> b) {
    Dual<K> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(Dual<K> a, Dual<K> b) {
    Dual<K> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(Dual<K> a, double b) { a.v += b; return a; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(Dual<K> a, double b) { a.v -= b; return a; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(double a, Dual<K> b) {
    b.v = a - b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) b.d[i] = -b.d[i];
    return b;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(double a, Dual<K> b) {
    b.v *= a;
#pragma unroll
    for (int i = 0; i < K; ++i) b.d[i] *= a;
    return b;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(Dual<K> a, double b) {
    const double ib = 1.0 / b;
    a.v *= ib;
#pragma unroll
    for (int i = 0; i < K; ++i) a.d[i] *= ib;
    return a;
}
template <int K>
__device__ __forceinline__ Dual<K> dsqrt(Dual<K> a) {
    Dual<K> r;
    r.v = sqrt(a.v);
    const double h = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * h;
    return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dmax(Dual<K> a, Dual<K> b) { return a.v >= b.v ? a : b; }

// ---------------------------------------------------------------- the law
// W(chi / scale), W(x) = max(0, 1 - x); a zero scale is fully softened
template <int K>
__device__ __forceinline__ Dual<K> soft(double scale, Dual<K> chi) {
    if (!(scale > 0.0)) return cst<K>(0.0);
    const Dual<K> x = chi / scale;
    return x.v >= 1.0 ? cst<K>(0.0) : 1.0 - x;
}
template <int K>
__device__ __forceinline__ Dual<K> friction(const Prm& P, Dual<K> chis) {
    return (P.fp - P.fr) * soft(P.dc, chis) + P.fr;
}
template <int K>
__device__ __forceinline__ Dual<K> dilatancy(const Prm& P, Dual<K> chis) { return P.psip * soft(P.dc, chis); }
template <int K>
__device__ __forceinline__ Dual<K> cohesion(const Prm& P, Dual<K> chit) { return P.cp * soft(P.wc, chit); }
template <int K>
__device__ __forceinline__ Dual<K> tstrength(const Prm& P, Dual<K> chit) { return P.sigp * soft(P.wc, chit); }

template <int K>
__device__ __forceinline__ Dual<K> norm2(Dual<K> a, Dual<K> b) { return dsqrt(a * a + b * b); }
template <int K>
__device__ __forceinline__ Dual<K> norm3(Dual<K> a, Dual<K> b, Dual<K> c) { return dsqrt(a * a + b * b + c * c); }

// state at t^n of one point (values) and its trial quantities (duals in Delta delta)
struct Pt {
    double T[3], dp[3], chis, chit, wdil;
};

template <int K>
struct Res {
    Dual<K> T[3], dp[3], chis, chit, wdil;
    int32_t mode;
};

// The three multiplier equations g(dl) = 0 of the returns, on duals of the trial
// quantities (K components) and of dl.  `aux` receives the state at that dl.
// Coulomb return (flow along s_hat + psi n, shear direction of the trial kept)
template <int K>
struct CoulombEq {
    const Prm* P;
    Dual<K> Ttr_n, tau_tr, s0, s1;
    double dp[3], chis, chit;
    __device__ Dual<K> g(Dual<K> dl, Res<K>* out) const {
        const Dual<K> dps0 = cst<K>(dp[0]) + dl * s0, dps1 = cst<K>(dp[1]) + dl * s1;
        const Dual<K> chis1 = dmax(cst<K>(chis), norm2(dps0, dps1));
        const Dual<K> psi1 = dilatancy(*P, chis1);
        const Dual<K> dpn = cst<K>(dp[2]) + dl * psi1;
        const Dual<K> chit1 = dmax(cst<K>(chit), norm3(dps0, dps1, dpn));
        const Dual<K> tau1 = tau_tr - P->Ks * dl;
        const Dual<K> Tn1 = Ttr_n - P->Kn * (psi1 * dl);
        if (out) {
            out->T[0] = tau1 * s0;
            out->T[1] = tau1 * s1;
            out->T[2] = Tn1;
            out->dp[0] = dps0;
            out->dp[1] = dps1;
            out->dp[2] = dpn;
            out->chis = chis1;
            out->chit = chit1;
            out->wdil = psi1 * dl;  // increment; the caller adds w_dil^n
        }
        return tau1 + friction(*P, chis1) * Tn1 - cohesion(*P, chit1);
    }
};

// tensile return (flow along n)
template <int K>
struct TensileEq {
    const Prm* P;
    Dual<K> Ttr_n;
    double dp[3], chit;
    __device__ Dual<K> g(Dual<K> dl, Res<K>* out) const {
        const Dual<K> dpn = cst<K>(dp[2]) + dl;
        const Dual<K> chit1 = dmax(cst<K>(chit), norm3(cst<K>(dp[0]), cst<K>(dp[1]), dpn));
        const Dual<K> Tn1 = Ttr_n - P->Kn * dl;
        if (out) {
            out->T[2] = Tn1;
            out->dp[2] = dpn;
            out->chit = chit1;
        }
        return Tn1 - tstrength(*P, chit1);
    }
};

// apex of the Coulomb cone: shear fully inelastic, normal increment mu
template <int K>
struct ApexEq {
    const Prm* P;
    Dual<K> Ttr_n, f1, dps0, dps1;
    double dpn, chit;
    __device__ Dual<K> g(Dual<K> mu, Res<K>* out) const {
        const Dual<K> dpn1 = cst<K>(dpn) + mu;
        const Dual<K> chit1 = dmax(cst<K>(chit), norm3(dps0, dps1, dpn1));
        const Dual<K> Tn1 = Ttr_n - P->Kn * mu;
        if (out) {
            out->T[2] = Tn1;
            out->dp[2] = dpn1;
            out->chit = chit1;
        }
        return f1 * Tn1 - cohesion(*P, chit1);
    }
};

// Root of g on [0, hi] with g(0) > 0 >= g(hi) (values), 0 when g(0) <= 0: Newton from 0
// safeguarded by the bracket -- a bisection step replaces the Newton step when that
// would leave the bracket or would not at least halve the step before last (the rule of
// the safeguarded Newton method of Press et al., Numerical Recipes, "rtsafe"); converged
// when a step is below 1e-16 of the iterate.  `Eq1` is the equation on one-component
// duals (the derivative in dl).
// x0: a first guess inside (0, hi) (the multiplier without softening), else 0.
template <class Eq1>
__device__ double find_root(const Eq1& e, double hi, double x0, int* st) {
    Dual<1> z;
    z.v = 0.0;
    z.d[0] = 1.0;
    Dual<1> gz = e.g(z, nullptr);
    if (!(gz.v > 0.0)) return 0.0;
    double lo = 0.0, x = 0.0, dx = hi, dxold = hi;
    if (x0 > 0.0 && x0 < hi) {
        x = x0;
        z.v = x;
        gz = e.g(z, nullptr);
    }
    for (int it = 0; it < 200; ++it) {
        // gz = g(x); the bracket keeps g(lo) > 0 >= g(hi)
        if (gz.v > 0.0) lo = x; else hi = x;
        if (gz.v == 0.0) return x;
        const double gp = gz.d[0];
        const double xn = x - gz.v / gp;
        if (!(gp < 0.0) || !(xn > lo && xn < hi) || fabs(2.0 * gz.v) > fabs(dxold * gp)) {
            dxold = dx;
            dx = 0.5 * (hi - lo);
            x = lo + dx;
            if (x == lo || x == hi) return x;
        } else {
            dxold = dx;
            dx = x - xn;
            x = xn;
        }
        if (fabs(dx) <= 1e-16 * fabs(x) || !(hi > lo)) return x;
        z.v = x;
        gz = e.g(z, nullptr);
    }
    *st |= ST_NOROOT;
    return x;
}

// the multiplier as a dual in Delta delta: one Newton step at the root with the
// derivative in dl carried in a fourth component
template <class Eq4>
__device__ Dual<3> root_dual(const Eq4& e4, double x, int* st) {
    Dual<4> z = cst<4>(x);
    z.d[3] = 1.0;
    const Dual<4> g = e4.g(z, nullptr);
    Dual<3> r;
    if (!(g.d[3] != 0.0)) {
        *st |= ST_NOROOT;
        r = cst<3>(x);
        return r;
    }
    r.v = x;  // the root found in values; the step only supplies the derivative
#pragma unroll
    for (int i = 0; i < 3; ++i) r.d[i] = -g.d[i] / g.d[3];
    return r;
}

template <int KA, int KB>
__device__ __forceinline__ Dual<KB> widen(Dual<KA> a) {
    Dual<KB> r;
    r.v = a.v;
#pragma unroll
    for (int i = 0; i < KB; ++i) r.d[i] = i < KA ? a.d[i] : 0.0;
    return r;
}

// open state: T' = 0, all of dd + C^-1 T'^n inelastic
template <int K>
__device__ void open_state(const Prm& P, const Pt& p, const Dual<K>* dd, Res<K>& r) {
    r.dp[0] = cst<K>(p.dp[0] + p.T[0] / P.Ks) + dd[0];
    r.dp[1] = cst<K>(p.dp[1] + p.T[1] / P.Ks) + dd[1];
    r.dp[2] = cst<K>(p.dp[2] + p.T[2] / P.Kn) + dd[2];
    r.T[0] = r.T[1] = r.T[2] = cst<K>(0.0);
    r.chis = dmax(cst<K>(p.chis), norm2(r.dp[0], r.dp[1]));
    r.chit = dmax(cst<K>(p.chit), norm3(r.dp[0], r.dp[1], r.dp[2]));
    r.wdil = cst<K>(p.wdil);
    r.mode = M_OPEN;
}

// the equations of one return on duals of K components, from the trial traction
template <int K>
__device__ CoulombEq<K> make_coulomb(const Prm& P, const Dual<K>* Ttr, const double* dpb, const Pt& p) {
    CoulombEq<K> e;
    e.P = &P;
    e.tau_tr = norm2(Ttr[0], Ttr[1]);
    e.s0 = Ttr[0] / e.tau_tr;
    e.s1 = Ttr[1] / e.tau_tr;
    e.Ttr_n = Ttr[2];
    e.dp[0] = dpb[0];
    e.dp[1] = dpb[1];
    e.dp[2] = dpb[2];
    e.chis = p.chis;
    e.chit = p.chit;
    return e;
}

template <int K>
__device__ ApexEq<K> make_apex(const Prm& P, const Dual<K>* Ttr, const double* dpb, const Pt& p) {
    ApexEq<K> e;
    e.P = &P;
    const Dual<K> tau = norm2(Ttr[0], Ttr[1]);
    if (tau.v > 0.0) {
        e.dps0 = cst<K>(dpb[0]) + Ttr[0] / P.Ks;
        e.dps1 = cst<K>(dpb[1]) + Ttr[1] / P.Ks;
    } else {
        e.dps0 = cst<K>(dpb[0]);
        e.dps1 = cst<K>(dpb[1]);
    }
    e.f1 = friction(P, dmax(cst<K>(p.chis), norm2(e.dps0, e.dps1)));
    e.Ttr_n = Ttr[2];
    e.dpn = dpb[2];
    e.chit = p.chit;
    return e;
}

template <int K>
__device__ TensileEq<K> make_tensile(const Prm& P, const Dual<K>* Ttr, const double* dpb, const Pt& p) {
    TensileEq<K> e;
    e.P = &P;
    e.Ttr_n = Ttr[2];
    e.dp[0] = dpb[0];
    e.dp[1] = dpb[1];
    e.dp[2] = dpb[2];
    e.chit = p.chit;
    return e;
}

// trial traction with the closed-state reference (damaged) or the plain one
template <int K>
__device__ void trial(const Prm& P, const Pt& p, const Dual<K>* dd, double dpn_shift, Dual<K>* Ttr) {
    Ttr[0] = cst<K>(p.T[0]) + P.Ks * dd[0];
    Ttr[1] = cst<K>(p.T[1]) + P.Ks * dd[1];
    Ttr[2] = cst<K>(p.T[2] - P.Kn * dpn_shift) + P.Kn * dd[2];
}

// The active mode at the trial state (values only; reading of the mode rules with
// hm_interface_update in hmat.h): M_ELASTIC, M_COULOMB, M_TENSILE, M_OPEN or M_APEX (a
// Coulomb return without a root before the shear traction vanishes).  dpb: the inelastic
// DD the return starts from (the closed-state normal part of a damaged point); shift:
// its normal change.
// the inelastic DD a return starts from and its normal change (closed-state reference of
// a fully damaged point); true if the point is fully damaged
__device__ __forceinline__ bool start_state(const Prm& P, const Pt& p, double dpb[3], double& shift) {
    const bool damaged = !(P.wc > 0.0) || p.chit >= P.wc;
    dpb[0] = p.dp[0];
    dpb[1] = p.dp[1];
    dpb[2] = p.dp[2];
    shift = 0.0;
    if (damaged) {
        const double wR = P.alphaR * P.wc + p.wdil;
        const double dpn_c = fmin(p.dp[2], wR);
        shift = dpn_c - p.dp[2];
        dpb[2] = dpn_c;
    }
    return damaged;
}

__device__ int classify(const Prm& P, const Pt& p, const double ddv[3], double dpb[3], double& shift) {
    const bool damaged = start_state(P, p, dpb, shift);
    Dual<1> dd1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dd1[i] = cst<1>(ddv[i]);
    int kind;
    if (damaged) {
        Dual<1> Ttr[3];
        trial(P, p, dd1, shift, Ttr);
        if (Ttr[2].v > 0.0) return M_OPEN;
        const double Fc = sqrt(Ttr[0].v * Ttr[0].v + Ttr[1].v * Ttr[1].v) +
                          friction(P, cst<1>(p.chis)).v * Ttr[2].v;  // no cohesion left
        kind = Fc <= 0.0 ? M_ELASTIC : M_COULOMB;
    } else {
        Dual<1> Ttr[3];
        trial(P, p, dd1, 0.0, Ttr);
        const double tau = sqrt(Ttr[0].v * Ttr[0].v + Ttr[1].v * Ttr[1].v);
        const double f0 = friction(P, cst<1>(p.chis)).v, c0 = cohesion(P, cst<1>(p.chit)).v,
                     st0 = tstrength(P, cst<1>(p.chit)).v;
        const double Fc = tau + f0 * Ttr[2].v - c0, Ft = Ttr[2].v - st0;
        if (Fc <= 0.0 && Ft <= 0.0) return M_ELASTIC;
        const double a = sqrt(1.0 + f0 * f0) - f0;
        const double h = tau - (c0 - f0 * st0) - a * (Ttr[2].v - st0);
        kind = h > 0.0 ? M_COULOMB : M_TENSILE;
    }
    if (kind == M_COULOMB) {
        Dual<1> Ttr[3];
        trial(P, p, dd1, shift, Ttr);
        const double tau = norm2(Ttr[0], Ttr[1]).v;
        if (!(tau > 0.0)) return M_APEX;
        const CoulombEq<1> e1 = make_coulomb<1>(P, Ttr, dpb, p);
        if (e1.g(cst<1>(tau / P.Ks), nullptr).v > 0.0) return M_APEX;
    }
    return kind;
}

// The return of the given mode on three-component duals (derivatives in Delta delta);
// with want_dual false the multipliers' derivative steps are skipped (values only).
__device__ Res<3> finish(const Prm& P, const Pt& p, const double ddv[3], int kind, const double dpb[3],
                         double shift, bool want_dual, int* st) {
    Dual<3> dd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dd[i] = cst<3>(ddv[i]);
        if (want_dual) dd[i].d[i] = 1.0;
    }
    Res<3> r;
    if (kind == M_OPEN) {
        open_state(P, p, dd, r);
        return r;
    }
    Dual<3> Ttr[3];
    trial(P, p, dd, shift, Ttr);
    if (kind == M_ELASTIC) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r.T[i] = Ttr[i];
            r.dp[i] = cst<3>(dpb[i]);
        }
        r.chis = cst<3>(p.chis);
        r.chit = cst<3>(p.chit);
        r.wdil = cst<3>(p.wdil);
        r.mode = M_ELASTIC;
        return r;
    }
    // the same trial on one- and four-component duals (values only in the first, dd in
    // the first three components of the second)
    Dual<1> T1[3];
    Dual<4> T4[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T1[i] = cst<1>(Ttr[i].v);
        T4[i] = widen<3, 4>(Ttr[i]);
    }
    if (kind == M_COULOMB) {
        const double tau = norm2(Ttr[0], Ttr[1]).v;
        const CoulombEq<1> e1 = make_coulomb<1>(P, T1, dpb, p);
        // without softening the multiplier is F_trial / (Ks + f psi Kn)
        const double f0 = friction(P, cst<1>(p.chis)).v, psi0 = dilatancy(P, cst<1>(p.chis)).v;
        const double F0 = tau + f0 * Ttr[2].v - cohesion(P, cst<1>(p.chit)).v;
        const double x = find_root(e1, tau / P.Ks, F0 / (P.Ks + f0 * psi0 * P.Kn), st);
        Dual<3> dl = cst<3>(x);
        if (want_dual && x > 0.0) dl = root_dual(make_coulomb<4>(P, T4, dpb, p), x, st);
        const CoulombEq<3> e3 = make_coulomb<3>(P, Ttr, dpb, p);
        Res<3> s;
        e3.g(dl, &s);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r.T[i] = s.T[i];
            r.dp[i] = s.dp[i];
        }
        r.chis = s.chis;
        r.chit = s.chit;
        r.wdil = cst<3>(p.wdil) + s.wdil;
        r.mode = M_COULOMB;
        return r;  // a Coulomb return stays in contact whatever the damage
    }
    if (kind == M_APEX) {
        const ApexEq<1> e1 = make_apex<1>(P, T1, dpb, p);
        const double x = find_root(e1, Ttr[2].v / P.Kn,
                                   e1.f1.v > 0.0 ? (Ttr[2].v - cohesion(P, cst<1>(p.chit)).v / e1.f1.v) / P.Kn : 0.0,
                                   st);
        Dual<3> mu = cst<3>(x);
        if (want_dual && x > 0.0) mu = root_dual(make_apex<4>(P, T4, dpb, p), x, st);
        const ApexEq<3> e3 = make_apex<3>(P, Ttr, dpb, p);
        Res<3> s;
        e3.g(mu, &s);
        r.T[0] = r.T[1] = cst<3>(0.0);
        r.T[2] = s.T[2];
        r.dp[0] = e3.dps0;
        r.dp[1] = e3.dps1;
        r.dp[2] = s.dp[2];
        r.chis = dmax(cst<3>(p.chis), norm2(e3.dps0, e3.dps1));
        r.chit = s.chit;
        r.mode = M_APEX;
    } else {
        const TensileEq<1> e1 = make_tensile<1>(P, T1, dpb, p);
        const double x = find_root(e1, Ttr[2].v / P.Kn, (Ttr[2].v - tstrength(P, cst<1>(p.chit)).v) / P.Kn, st);
        Dual<3> dl = cst<3>(x);
        if (want_dual && x > 0.0) dl = root_dual(make_tensile<4>(P, T4, dpb, p), x, st);
        const TensileEq<3> e3 = make_tensile<3>(P, Ttr, dpb, p);
        Res<3> s;
        e3.g(dl, &s);
        r.T[0] = Ttr[0];
        r.T[1] = Ttr[1];
        r.T[2] = s.T[2];
        r.dp[0] = cst<3>(dpb[0]);
        r.dp[1] = cst<3>(dpb[1]);
        r.dp[2] = s.dp[2];
        r.chis = cst<3>(p.chis);
        r.chit = s.chit;
        r.mode = M_TENSILE;
    }
    r.wdil = cst<3>(p.wdil);
    if (!(P.wc > 0.0) || r.chit.v >= P.wc) open_state(P, p, dd, r);  // full damage: open
    return r;
}

struct IfArgs {
    Prm P;
    int64_t n;
    const double *T, *dp, *chi, *dd;  // the outputs may alias these: a point is read before it is written
    double *T1, *dp1, *chi1, *cep;
    int32_t* mode;
    unsigned long long* counts;  // per mode, then unresolved (or NULL)
    int32_t* list;               // [3][n]: points of the Coulomb, tensile and apex returns
    unsigned int* lcount;        // [3]
};

__device__ __forceinline__ void load_point(const IfArgs& a, int64_t e, Pt& p, double ddv[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p.T[i] = a.T[3 * e + i];
        p.dp[i] = a.dp[3 * e + i];
        ddv[i] = a.dd[3 * e + i];
    }
    p.chis = a.chi[3 * e];
    p.chit = a.chi[3 * e + 1];
    p.wdil = a.chi[3 * e + 2];
}

__device__ __forceinline__ void store_point(const IfArgs& a, int64_t e, const Res<3>& r, int st,
                                            unsigned int* s_cnt) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        a.T1[3 * e + i] = r.T[i].v;
        a.dp1[3 * e + i] = r.dp[i].v;
    }
    a.chi1[3 * e] = r.chis.v;
    a.chi1[3 * e + 1] = r.chit.v;
    a.chi1[3 * e + 2] = r.wdil.v;
    if (a.cep) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) a.cep[9 * e + 3 * i + j] = r.T[i].d[j];
    }
    if (a.mode) a.mode[e] = r.mode | (st ? 256 : 0);
    atomicAdd(&s_cnt[r.mode], 1u);
    if (st) atomicAdd(&s_cnt[N_MODES], 1u);
}

__device__ __forceinline__ void flush_counts(const IfArgs& a, unsigned int* s_cnt) {
    __syncthreads();
    if (a.counts && threadIdx.x < N_MODES + 1 && s_cnt[threadIdx.x])
        atomicAdd(&a.counts[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
}

// list slot of each return kind (Coulomb, tensile, apex)
__device__ __forceinline__ int list_of(int kind) {
    return kind == M_COULOMB ? 0 : (kind == M_TENSILE ? 1 : (kind == M_APEX ? 2 : -1));
}

// Pass 1, one thread per point: the mode; elastic and open points are finished here, the
// returns are listed by kind so that pass 2 runs each kind in warps of that kind only
// (a warp over mixed modes would run every branch).
__global__ void __launch_bounds__(128) k_iface_classify(IfArgs a) {
    __shared__ unsigned int s_cnt[N_MODES + 1];
    if (threadIdx.x < N_MODES + 1) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int kind = -1;
    Pt p;
    double ddv[3], dpb[3], shift = 0.0;
    if (e < a.n) {
        load_point(a, e, p, ddv);
        kind = classify(a.P, p, ddv, dpb, shift);
        if (kind == M_ELASTIC || kind == M_OPEN) {
            int st = 0;
            store_point(a, e, finish(a.P, p, ddv, kind, dpb, shift, a.cep != nullptr, &st), st, s_cnt);
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, list_of(kind) == k);
        if (m == 0u) continue;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&a.lcount[k], (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (list_of(kind) == k) a.list[(int64_t)k * a.n + base + __popc(m & ((1u << lane) - 1u))] = (int32_t)e;
    }
    flush_counts(a, s_cnt);
}

// Pass 2: the listed points of one return kind, grid-stride
__global__ void __launch_bounds__(128) k_iface_return(IfArgs a, int k) {
    __shared__ unsigned int s_cnt[N_MODES + 1];
    if (threadIdx.x < N_MODES + 1) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int kind = k == 0 ? M_COULOMB : (k == 1 ? M_TENSILE : M_APEX);
    const int64_t cnt = a.lcount[k];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = a.list[(int64_t)k * a.n + q];
        Pt p;
        double ddv[3], dpb[3], shift = 0.0;
        load_point(a, e, p, ddv);
        start_state(a.P, p, dpb, shift);
        int st = 0;
        store_point(a, e, finish(a.P, p, ddv, kind, dpb, shift, a.cep != nullptr, &st), st, s_cnt);
    }
    flush_counts(a, s_cnt);
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }
bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

}  // namespace
}  // namespace hm

extern "C" hm_status hm_interface_update(const hm_interface_params* prm, int64_t n, const double* T_dev,
                                         const double* dp_dev, const double* chi_dev, const double* dd_dev,
                                         double* T1_dev, double* dp1_dev, double* chi1_dev, double* cep_dev,
                                         int32_t* mode_dev, int64_t* counts, void* stream) {
    using namespace hm;
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_interface_update");
    if (!prm) fail(HM_EINVAL, "interface_update: params is NULL");
    if (n < 0) fail(HM_EINVAL, "interface_update: n < 0");
    const hm_interface_params& q = *prm;
    if (!finite_pos(q.Ks) || !finite_pos(q.Kn)) fail(HM_EINVAL, "interface_update: stiffnesses must be > 0");
    if (!finite_nonneg(q.fp) || !finite_nonneg(q.fr) || !finite_nonneg(q.psip) || !finite_nonneg(q.cp) ||
        !finite_nonneg(q.sigp) || !finite_nonneg(q.wc) || !finite_nonneg(q.alphaR))
        fail(HM_EINVAL, "interface_update: friction, dilatancy, strengths, w_c and alpha_R must be finite and >= 0");
    if (!(q.dc > 0.0) || std::isnan(q.dc)) fail(HM_EINVAL, "interface_update: d_c must be > 0");
    if (n > 0 && (!T_dev || !dp_dev || !chi_dev || !dd_dev || !T1_dev || !dp1_dev || !chi1_dev))
        fail(HM_EINVAL, "interface_update: a state or increment pointer is NULL");
    if (n > INT32_MAX) fail(HM_EINVAL, "interface_update: more than 2^31 - 1 points");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf<unsigned long long> cnt;
    if (counts) {
        cnt.alloc(N_MODES + 1);
        HM_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), st));
    }
    const Prm P{q.Ks, q.Kn, q.fp, q.fr, q.psip, q.dc, q.cp, q.sigp, q.wc, q.alphaR};
    if (n > 0) {
        // stream-ordered scratch for the per-kind lists: no device-wide synchronisation
        void* scratch = nullptr;
        const size_t lbytes = (size_t)3 * n * sizeof(int32_t), cbytes = 4 * sizeof(unsigned int);
        HM_CUDA(cudaMallocAsync(&scratch, lbytes + cbytes, st));
        IfArgs a{P, n, T_dev, dp_dev, chi_dev, dd_dev, T1_dev, dp1_dev, chi1_dev, cep_dev, mode_dev,
                 counts ? cnt.p : nullptr, (int32_t*)scratch, (unsigned int*)((char*)scratch + lbytes)};
        cudaError_t err = cudaMemsetAsync(a.lcount, 0, cbytes, st);
        if (err == cudaSuccess) {
            k_iface_classify<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(a);
            int dev = 0, nsm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            const unsigned g2 = (unsigned)std::min<int64_t>(ceil_div(n, 128), (int64_t)std::max(nsm, 1) * 16);
            for (int k = 0; k < 3; ++k) k_iface_return<<<g2, 128, 0, st>>>(a, k);
            err = cudaGetLastError();
        }
        HM_CUDA(cudaFreeAsync(scratch, st));
        HM_CUDA(err);
    }
    if (counts) {
        unsigned long long h[N_MODES + 1];
        HM_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i <= N_MODES; ++i) counts[i] = (int64_t)h[i];
        if (h[N_MODES]) fail(HM_ENOCONV, "interface_update: a plastic multiplier did not converge (" +
                                             std::to_string(h[N_MODES]) + " points)");
    }
    HM_API_END
}
