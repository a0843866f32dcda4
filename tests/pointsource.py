"""Independent brute-force reference for the pins: the stress of a point displacement
discontinuity from Kelvin's solution, integrated numerically over a rectangle.

Nothing here is shared with the oracle or the CUDA path.  A DD b on an area element dA
with unit normal nu acts as the moment tensor M_pq = dA [lam (b.nu) d_pq + mu (b_p nu_q +
b_q nu_p)] (delta = u+ - u-, nu from the minus to the plus face), whose displacement is
u_k(x) = -M_pq d/dx_q G_kp(x - y) with Kelvin's tensor
G_kp(r) = [(3 - 4 v) d_kp / |r| + r_k r_p / |r|^3] / (16 pi mu (1 - v)).
"""
from __future__ import annotations

import math

import numpy as np

I3 = np.eye(3)


def kelvin_d2(r, mu, nu):
    """d^2 G_kp / dx_j dx_q at separation vectors r (..., 3) -> (..., k, p, q, j)."""
    R = np.linalg.norm(r, axis=-1)[..., None, None, None, None]
    rk = r[..., :, None, None, None]
    rp = r[..., None, :, None, None]
    rq = r[..., None, None, :, None]
    rj = r[..., None, None, None, :]
    dkp = I3[:, :, None, None]
    dqj = I3[None, None, :, :]
    dkq = I3[:, None, :, None]
    dpj = I3[None, :, None, :]
    dkj = I3[:, None, None, :]
    dpq = I3[None, :, :, None]
    # second derivative of 1/r:  -d_qj / r^3 + 3 r_q r_j / r^5
    t1 = dkp * (-dqj / R ** 3 + 3.0 * rq * rj / R ** 5)
    # second derivative of r_k r_p / r^3
    t2 = ((dkq * dpj + dkj * dpq) / R ** 3
          - 3.0 * (dkq * rp + rk * dpq) * rj / R ** 5
          - 3.0 * (dkj * rp * rq + rk * dpj * rq + rk * rp * dqj) / R ** 5
          + 15.0 * rk * rp * rq * rj / R ** 7)
    A = 1.0 / (16.0 * math.pi * mu * (1.0 - nu))
    return A * ((3.0 - 4.0 * nu) * t1 + t2)


def point_stress(x, y, nvec, bvec, mu, nu, dA):
    """Stress at x (3,) from point DDs at y (..., 3) with normal nvec and DD bvec, weights dA (...)."""
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    M = lam * np.dot(bvec, nvec) * I3 + mu * (np.outer(bvec, nvec) + np.outer(nvec, bvec))
    D = kelvin_d2(x[None, :] - y, mu, nu)  # (npts, k, p, q, j)
    grad = -np.einsum("pq,nkpqj,n->kj", M, D, dA)  # u_{k,j}
    th = np.trace(grad)
    return lam * th * I3 + mu * (grad + grad.T)


_GL = {}


def _gauss(n):
    if n not in _GL:
        _GL[n] = np.polynomial.legendre.leggauss(n)
    return _GL[n]


def rect_stress(x, c, s1, s2, nvec, a, b, bvec, mu, nu, order=10, rel=1e-13, depth=0, box=None):
    """Adaptive tensor Gauss-Legendre integral of the point stress over the rectangle
    c + xi s1 + eta s2, |xi| <= a, |eta| <= b (bvec in global components)."""
    if box is None:
        box = (-a, a, -b, b)
    x0, x1, y0, y1 = box

    def panel(bx):
        u0, u1, v0, v1 = bx
        g, w = _gauss(order)
        xi = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * g
        et = 0.5 * (v0 + v1) + 0.5 * (v1 - v0) * g
        XI, ET = np.meshgrid(xi, et, indexing="ij")
        W = np.outer(w, w) * 0.25 * (u1 - u0) * (v1 - v0)
        pts = c[None, :] + XI.ravel()[:, None] * s1[None, :] + ET.ravel()[:, None] * s2[None, :]
        return point_stress(x, pts, nvec, bvec, mu, nu, W.ravel())

    whole = panel(box)
    xm, ym = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
    kids = [(x0, xm, y0, ym), (xm, x1, y0, ym), (x0, xm, ym, y1), (xm, x1, ym, y1)]
    parts = [panel(k) for k in kids]
    tot = sum(parts)
    scale = max(np.abs(tot).max(), 1e-300)
    if np.abs(tot - whole).max() <= rel * scale or depth >= 14:
        return tot
    return sum(rect_stress(x, c, s1, s2, nvec, a, b, bvec, mu, nu, order, rel, depth + 1, k) for k in kids)


def brute_block(xr, rframe, cs, sframe, a, b, E, nu, rel=1e-12):
    """3x3 block by quadrature: traction (receiver frame) from unit DD components
    (source frame)."""
    mu = E / (2.0 * (1.0 + nu))
    out = np.zeros((3, 3))
    for m in range(3):
        sig = rect_stress(np.asarray(xr, float), np.asarray(cs, float), np.asarray(sframe[0], float),
                          np.asarray(sframe[1], float), np.asarray(sframe[2], float), a, b,
                          np.asarray(sframe[m], float), mu, nu, rel=rel)
        t = sig @ np.asarray(rframe[2], float)
        for al in range(3):
            out[al, m] = np.dot(rframe[al], t)
    return out


def point_block(xr, rframe, cs, sframe, area, E, nu):
    """Far-field approximation: the whole rectangle lumped into one point DD."""
    mu = E / (2.0 * (1.0 + nu))
    out = np.zeros((3, 3))
    for m in range(3):
        sig = point_stress(np.asarray(xr, float), np.asarray(cs, float)[None, :], np.asarray(sframe[2], float),
                           np.asarray(sframe[m], float), mu, nu, np.array([area]))
        t = sig @ np.asarray(rframe[2], float)
        for al in range(3):
            out[al, m] = np.dot(rframe[al], t)
    return out


def coplanar_closed_form(x1, x2, a, b, E, nu):
    """Receiver in the plane of the source (same frame): traction from unit DDs by the
    corner formulas of the planar-crack finite-part integrals, C = mu / (4 pi (1 - nu)):
      normal:  t_n = C I3 delta_n,  I3 = sum_corners s (-R / (u v)),
      shear:   t_a = C [(1 - 2 nu) I3 delta_a + nu (D_ab + d_ab I3) delta_b],
               D_11 = sum s (-v / (u R)), D_22 = sum s (-u / (v R)), D_12 = sum s (1 / R);
    normal and shear are uncoupled."""
    mu = E / (2.0 * (1.0 + nu))
    C = mu / (4.0 * math.pi * (1.0 - nu))
    I3v = D11 = D22 = D12 = 0.0
    for su in (1.0, -1.0):
        for sv in (1.0, -1.0):
            s = su * sv
            u = x1 + su * a
            v = x2 + sv * b
            R = math.hypot(u, v)
            I3v += s * (-R / (u * v))
            D11 += s * (-v / (u * R))
            D22 += s * (-u / (v * R))
            D12 += s * (1.0 / R)
    D = np.array([[D11, D12], [D12, D22]])
    out = np.zeros((3, 3))
    out[2, 2] = C * I3v
    for al in range(2):
        for be in range(2):
            out[al, be] = C * ((1.0 - 2.0 * nu) * I3v * (al == be) + nu * (D[al, be] + (al == be) * I3v))
    return out
