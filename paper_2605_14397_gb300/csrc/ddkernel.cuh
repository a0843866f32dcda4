// Device evaluation of one 3x3 influence block of the collocation DD matrix E.
//
// Block (i, j): traction at the centroid of element i (components on its frame
// s1, s2, n) from a unit DD component constant over element j -- a rectangle or a
// triangle -- (components on j's frame), full-space isotropic elasticity (Sec. 3.1,
// eq. TractionBIE-general reduced to the fracture integral; eq. ElasSystem).
//
// Formulation used here.  In source-local coordinates (source plane x3 = 0) the stress
// of a unit DD along local axis m is, with phi(x) = int int_rect 1/R,
// C = mu / (4 pi (1 - nu)) and P_.. the derivatives of phi,
//   sigma^(m)_kj = -C [ 2 nu d_kj P_3m + (1-nu)(d_km P_3j + d_jm P_3k)
//                      - (1-2nu) d_m3 P_kj - nu (d_k3 P_mj + d_j3 P_mk) - x3 P_mkj ].
// (Moment tensor of a DD on Kelvin's solution, integrated over the rectangle.)
// phi's second and third derivatives are corner sums of rational functions of
// (u, v, x3, R); phi is even in every coordinate, so they are evaluated at |x| where
// the corners at positive u/v take the direct forms and the others the rationalised
// ones 1/(v+R) = (R-v)/(u^2+x3^2) -- no cancellation between corner terms of one edge.
// All arithmetic is FP64.
#pragma once

#include "common.h"

namespace hm {

struct PhiDerivs {
    // second derivatives
    double d11, d22, d12, d13, d23, d33;
    // third derivatives (10 distinct)
    double d111, d112, d122, d222, d113, d123, d223, d133, d233, d333;
};

// Returns false if the point lies on the rectangle boundary (in-plane, within tol).
__device__ __forceinline__ bool phi_corner_sums(double x1, double x2, double x3, double a, double b,
                                                double tol, PhiDerivs& D) {
    const double g1 = x1 < 0.0 ? -1.0 : 1.0;
    const double g2 = x2 < 0.0 ? -1.0 : 1.0;
    const double g3 = x3 < 0.0 ? -1.0 : 1.0;
    const double X = fabs(x1), Y = fabs(x2), Z = fabs(x3);
    if (Z <= tol && ((fabs(X - a) <= tol && Y <= b + tol) || (fabs(Y - b) <= tol && X <= a + tol)))
        return false;
    const double z2 = Z * Z;
    double s11 = 0, s22 = 0, s12 = 0, s13 = 0, s23 = 0;
    double t111 = 0, t112 = 0, t122 = 0, t222 = 0, t113 = 0, t123 = 0, t223 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double su = (c & 1) ? -1.0 : 1.0;
        const double sv = (c & 2) ? -1.0 : 1.0;
        const double sgn = su * sv;
        const double u = X + su * a;
        const double v = Y + sv * b;
        const double u2 = u * u, v2 = v * v;
        const double R = sqrt(u2 + v2 + z2);
        const double p = 1.0 / R;
        const double Av = v >= 0.0 ? 1.0 / (v + R) : (R - v) / (u2 + z2);
        const double Au = u >= 0.0 ? 1.0 / (u + R) : (R - u) / (v2 + z2);
        const double p2 = p * p, p3 = p2 * p;
        const double pAv = p * Av, pAu = p * Au;
        const double wv = p2 * Av * (p + Av);  // d/du of u p Av is p Av - u^2 wv
        const double wu = p2 * Au * (p + Au);
        s11 += sgn * u * pAv;
        s22 += sgn * v * pAu;
        s12 += sgn * p;
        s13 += sgn * Z * pAv;
        s23 += sgn * Z * pAu;
        t111 += sgn * (pAv - u2 * wv);
        t222 += sgn * (pAu - v2 * wu);
        t112 -= sgn * u * p3;
        t122 -= sgn * v * p3;
        t123 -= sgn * Z * p3;
        t113 -= sgn * u * Z * wv;
        t223 -= sgn * v * Z * wu;
    }
    // restore the signs: a derivative picks one sign factor per differentiated axis
    const double g12 = g1 * g2, g13 = g1 * g3, g23 = g2 * g3, g123 = g12 * g3;
    D.d11 = s11;
    D.d22 = s22;
    D.d33 = -(s11 + s22);
    D.d12 = g12 * s12;
    D.d13 = g13 * s13;
    D.d23 = g23 * s23;
    D.d111 = g1 * t111;
    D.d222 = g2 * t222;
    D.d112 = g2 * t112;
    D.d122 = g1 * t122;
    D.d113 = g3 * t113;
    D.d223 = g3 * t223;
    D.d123 = g123 * t123;
    D.d133 = -g1 * (t111 + t122);
    D.d233 = -g2 * (t112 + t222);
    D.d333 = -g3 * (t113 + t223);
    return true;
}

// The same derivatives for a triangle (vertices tv in the source plane frame, x3 = 0).
// Every derivative with an in-plane index alpha is, by Stokes' theorem, a sum over the
// edges of line integrals (d = x - xi, n the outward in-plane normal of the edge):
//   phi_{,alpha beta} = sum n_alpha int d_beta / R^3,
//   phi_{,alpha beta gamma} = -sum n_alpha int (3 d_beta d_gamma / R^5 - delta / R^3).
// Along an edge d = h + w tau, h perpendicular to the edge (in-plane part hp n and x3),
// w running from wB = wA - L to wA, R^2 = rho^2 + w^2; the integrals are the closed
// forms K3p = int w^p / R^3 and K5p = int w^p / R^5 written without 1/rho^2:
//   K30 = (wA^2 - wB^2) / (RA RB (wA RB + wB RA)) when wA, wB have one sign (else
//         (gA - gB) / rho^2, g = w / R), K31 = 1/RB - 1/RA, K51 = (1/RB^3 - 1/RA^3) / 3,
//   K52 = K30 (gA^2 + gA gB + gB^2) / 3,
//   K50 = K30 / 3 (1/RA^2 + 1/RB^2 + (1/RA^2 + 1/RB^2 - rho^2 / (RA RB)^2) / (1 + gA gB)),
// the last from K50 = (K30 - K52) / rho^2 and 1 - gA gB = (1 - gA^2 gB^2) / (1 + gA gB).
// The x3-x3 derivatives follow from Laplace's equation.  Returns false if the point
// lies on an edge (in-plane, within tol).
__device__ __forceinline__ bool phi_edge_sums(double x1, double x2, double x3, const double* tv, double tol,
                                              PhiDerivs& D) {
    const double o = (tv[2] - tv[0]) * (tv[5] - tv[1]) - (tv[3] - tv[1]) * (tv[4] - tv[0]);
    const int v1 = o < 0.0 ? 2 : 1, v2 = o < 0.0 ? 1 : 2;  // counter-clockwise order
    const double z = x3, z2 = z * z;
    double s11 = 0, s22 = 0, s12 = 0, s13 = 0, s23 = 0;
    double t111 = 0, t112 = 0, t122 = 0, t222 = 0, t113 = 0, t123 = 0, t223 = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int ia = e == 0 ? 0 : (e == 1 ? v1 : v2);
        const int ib = e == 0 ? v1 : (e == 1 ? v2 : 0);
        const double px = tv[2 * ia], py = tv[2 * ia + 1];
        const double ex = tv[2 * ib] - px, ey = tv[2 * ib + 1] - py;
        const double L = sqrt(ex * ex + ey * ey);
        const double tx = ex / L, ty = ey / L;
        const double nx = ty, ny = -tx;
        const double dx = x1 - px, dy = x2 - py;
        const double wA = dx * tx + dy * ty, wB = wA - L;
        const double hp = dx * nx + dy * ny;
        if (fabs(z) <= tol && fabs(hp) <= tol && wA >= -tol && wB <= tol) return false;
        const double rho2 = hp * hp + z2;
        const double RA = sqrt(rho2 + wA * wA), RB = sqrt(rho2 + wB * wB);
        const double gA = wA / RA, gB = wB / RB;
        const double K30 = wA * wB > 0.0 ? (wA * wA - wB * wB) / (RA * RB * (wA * RB + wB * RA)) : (gA - gB) / rho2;
        const double iA2 = 1.0 / (RA * RA), iB2 = 1.0 / (RB * RB);
        const double K31 = 1.0 / RB - 1.0 / RA;
        const double K51 = (iB2 / RB - iA2 / RA) / 3.0;
        const double K52 = K30 * (gA * gA + gA * gB + gB * gB) / 3.0;
        const double K50 = K30 / 3.0 * (iA2 + iB2 + (iA2 + iB2 - rho2 * iA2 * iB2) / (1.0 + gA * gB));
        const double h1 = hp * nx, h2 = hp * ny;
        const double I1 = h1 * K30 + tx * K31, I2 = h2 * K30 + ty * K31, I3 = z * K30;
        const double J11 = 3.0 * (h1 * h1 * K50 + 2.0 * h1 * tx * K51 + tx * tx * K52) - K30;
        const double J12 = 3.0 * (h1 * h2 * K50 + (h1 * ty + h2 * tx) * K51 + tx * ty * K52);
        const double J22 = 3.0 * (h2 * h2 * K50 + 2.0 * h2 * ty * K51 + ty * ty * K52) - K30;
        const double J13 = 3.0 * z * (h1 * K50 + tx * K51);
        const double J23 = 3.0 * z * (h2 * K50 + ty * K51);
        s11 += nx * I1;
        s12 += nx * I2;
        s13 += nx * I3;
        s22 += ny * I2;
        s23 += ny * I3;
        t111 -= nx * J11;
        t112 -= nx * J12;
        t122 -= nx * J22;
        t222 -= ny * J22;
        t113 -= nx * J13;
        t123 -= nx * J23;
        t223 -= ny * J23;
    }
    D.d11 = s11;
    D.d22 = s22;
    D.d33 = -(s11 + s22);
    D.d12 = s12;
    D.d13 = s13;
    D.d23 = s23;
    D.d111 = t111;
    D.d222 = t222;
    D.d112 = t112;
    D.d122 = t122;
    D.d113 = t113;
    D.d223 = t223;
    D.d123 = t123;
    D.d133 = -(t111 + t122);
    D.d233 = -(t112 + t222);
    D.d333 = -(t113 + t223);
    return true;
}

__device__ __forceinline__ double P2(const PhiDerivs& D, int i, int j) {
    // symmetric second-derivative lookup (indices are compile-time after unrolling)
    if (i > j) { int t = i; i = j; j = t; }
    if (i == 0) return j == 0 ? D.d11 : (j == 1 ? D.d12 : D.d13);
    if (i == 1) return j == 1 ? D.d22 : D.d23;
    return D.d33;
}

__device__ __forceinline__ double P3(const PhiDerivs& D, int i, int j, int k) {
    // sort the three indices
    if (i > j) { int t = i; i = j; j = t; }
    if (j > k) { int t = j; j = k; k = t; }
    if (i > j) { int t = i; i = j; j = t; }
    const int key = i * 9 + j * 3 + k;
    switch (key) {
        case 0: return D.d111;   // 000
        case 1: return D.d112;   // 001
        case 2: return D.d113;   // 002
        case 4: return D.d122;   // 011
        case 5: return D.d123;   // 012
        case 8: return D.d133;   // 022
        case 13: return D.d222;  // 111
        case 14: return D.d223;  // 112
        case 17: return D.d233;  // 122
        default: return D.d333;  // 222
    }
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Influence block of receiver element R from source element S; out[3*alpha + m].
// Returns false for a receiver on a source edge (out is NaN then).
__device__ __forceinline__ bool dd_block(const ElemRec& Rr, const ElemRec& Ss, double mu, double nu,
                                         double out[9]) {
    const double d[3] = {Rr.c[0] - Ss.c[0], Rr.c[1] - Ss.c[1], Rr.c[2] - Ss.c[2]};
    const double x1 = dot3(Ss.s1, d), x2 = dot3(Ss.s2, d), x3 = dot3(Ss.n, d);
    // receiver frame on source-local axes: q[alpha][k] = e_k(source) . e_alpha(receiver)
    double q[3][3];
    const double* re[3] = {Rr.s1, Rr.s2, Rr.n};
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        q[al][0] = dot3(Ss.s1, re[al]);
        q[al][1] = dot3(Ss.s2, re[al]);
        q[al][2] = dot3(Ss.n, re[al]);
    }
    PhiDerivs D;
    const bool ok = Ss.shape == HM_SHAPE_TRI ? phi_edge_sums(x1, x2, x3, Ss.tv, 1e-9 * sqrt(Ss.area), D)
                                              : phi_corner_sums(x1, x2, x3, Ss.a, Ss.b, 1e-9 * fmin(Ss.a, Ss.b), D);
    if (!ok) {
#pragma unroll
        for (int k = 0; k < 9; ++k) out[k] = __longlong_as_double(0x7ff8000000000000ULL);
        return false;
    }
    const double C = mu / (4.0 * 3.14159265358979323846 * (1.0 - nu));
    const double c_a = 2.0 * nu, c_b = 1.0 - nu, c_c = 1.0 - 2.0 * nu;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double sig[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int j = k; j < 3; ++j) {
                double s = 0.0;
                if (k == j) s += c_a * P2(D, 2, m);
                if (k == m) s += c_b * P2(D, 2, j);
                if (j == m) s += c_b * P2(D, 2, k);
                if (m == 2) s -= c_c * P2(D, k, j);
                if (k == 2) s -= nu * P2(D, m, j);
                if (j == 2) s -= nu * P2(D, m, k);
                s -= x3 * P3(D, m, k, j);
                sig[k][j] = -C * s;
                sig[j][k] = sig[k][j];
            }
        }
        // traction on the receiver plane, then on the receiver frame
        double t[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] = sig[k][0] * q[2][0] + sig[k][1] * q[2][1] + sig[k][2] * q[2][2];
#pragma unroll
        for (int al = 0; al < 3; ++al) out[3 * al + m] = q[al][0] * t[0] + q[al][1] * t[1] + q[al][2] * t[2];
    }
    return true;
}

}  // namespace hm
