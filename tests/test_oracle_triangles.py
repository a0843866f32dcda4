"""Pins of the oracle's triangle elements (Sec. 3.1: constant DD over triangles,
collocation at centroids), each against something other than the oracle's own edge
quadrature:

* a rectangle is two triangles: phi's second and third derivatives of the rectangle
  equal the sum over its two triangles at points in and off its plane (the shared
  diagonal's integrals cancel), and so does the whole 3x3 influence block;
* at a point inside a triangle, in its plane, the derivatives equal the finite parts
  written in polar coordinates about the point -- one-dimensional integrals over the
  angle of the distance to the boundary, an independent formula;
* off the plane they equal a brute-force two-dimensional quadrature over the triangle
  (collapsed Gauss rule), for general triangles;
* far away they tend to area x the derivatives of 1/r at the centroid;
* the dense operator of a triangulated penny crack gives Sneddon's opening, with the
  error falling as the mesh is refined.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import synth

E, NU = 1.0, 0.25


def tri_derivs(x, tv):
    st, d2, d3 = O.tri_phi_derivatives(x, tv)
    assert st == 0
    return d2, d3


def test_rectangle_is_two_triangles():
    a, b = 0.3, 0.2
    T1 = [(-a, -b), (a, -b), (a, b)]
    T2 = [(-a, -b), (a, b), (-a, b)]
    rng = np.random.default_rng(1)
    pts = []
    for z in (0.0, 1e-3, 0.05, 0.4, 3.0):
        for _ in range(12):
            p = rng.uniform(-0.6, 0.6, 2)
            # stay away from the edges, and in-plane from the shared diagonal
            if z == 0.0 and (min(abs(abs(p[0]) - a), abs(abs(p[1]) - b)) < 1e-2 or abs(p[0] * b - p[1] * a) < 1e-2):
                continue
            pts.append((p[0], p[1], z * rng.choice([-1.0, 1.0])))
    assert len(pts) > 40
    for x in pts:
        st, r2, r3 = O.phi_derivatives(x, a, b)
        assert st == 0
        a2, a3 = tri_derivs(x, T1)
        b2, b3 = tri_derivs(x, T2)
        assert np.abs(a2 + b2 - r2).max() <= 1e-12 * np.abs(r2).max(), x
        assert np.abs(a3 + b3 - r3).max() <= 1e-12 * np.abs(r3).max(), x


def test_rectangle_block_is_two_triangle_blocks():
    """The same at the level of the influence block, through global vertices and frames."""
    rng = np.random.default_rng(2)
    Q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    s1, s2, n = Q[:, 0], Q[:, 1], Q[:, 2]
    cs = np.array([0.1, -0.2, 0.3])
    a, b = 0.25, 0.15
    V = [cs + sa * a * s1 + sb * b * s2 for sa, sb in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    for _ in range(10):
        xr = cs + rng.normal(size=3) * 0.4
        R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        rf = (R[:, 0], R[:, 1], R[:, 2])
        st, Br = O.influence_point(xr, rf, cs, (s1, s2, n), a, b, E, NU)
        assert st == 0
        tot = np.zeros((3, 3))
        for tri in ((V[0], V[1], V[2]), (V[0], V[2], V[3])):
            # each triangle collocated at the rectangle's centre: only the integral moves
            st, Bt = O.influence_point_tri(xr, rf, cs, (s1, s2, n), np.array(tri), E, NU)
            assert st == 0
            tot += Bt
        assert np.abs(tot - Br).max() <= 1e-12 * np.abs(Br).max()


def _ray_distance(p, tv, th):
    """Distance from p (inside) along direction th to the triangle's boundary."""
    e = np.array([np.cos(th), np.sin(th)])
    best = np.inf
    for k in range(3):
        A, B = tv[k], tv[(k + 1) % 3]
        M = np.array([e, A - B]).T
        t, s = np.linalg.solve(M, A - p)
        if t > 0 and -1e-12 <= s <= 1 + 1e-12:
            best = min(best, t)
    return best


def _polar_finite_parts(p, tv, n=64):
    """phi's in-plane second and third derivatives and phi_33 at an interior point p of
    the triangle (in its plane), from the finite parts in polar coordinates about p:
    FP int_0^r rho^-2 d rho = -1/r and FP int_0^r rho^-3 d rho = -1/(2 r^2)."""
    ang = sorted(np.arctan2(v[1] - p[1], v[0] - p[0]) % (2 * np.pi) for v in tv)
    cuts = ang + [ang[0] + 2 * np.pi]
    xg, wg = np.polynomial.legendre.leggauss(n)
    d2 = np.zeros((3, 3))
    d3 = np.zeros((3, 3, 3))
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        for xi, wi in zip(xg, wg):
            th = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xi
            w = 0.5 * (hi - lo) * wi
            r = _ray_distance(p, tv, th)
            e = np.array([np.cos(th), np.sin(th)])
            for i, j in itertools.product(range(2), repeat=2):
                d2[i, j] += w * -(3 * e[i] * e[j] - (i == j)) / r
                for k in range(2):
                    dl = (i == j) * e[k] + (i == k) * e[j] + (j == k) * e[i]
                    d3[i, j, k] += w * (3 * dl - 15 * e[i] * e[j] * e[k]) / (2 * r * r)
            d2[2, 2] += w / r
    return d2, d3


@pytest.mark.parametrize("tv", [
    [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)],
    [(-0.4, -0.1), (0.5, -0.3), (0.1, 0.6)],
    [(0.0, 0.0), (2.0, 0.1), (0.3, 0.25)],  # obtuse and elongated
])
def test_interior_in_plane_values_are_the_polar_finite_parts(tv):
    tv = np.array(tv, dtype=float)
    for wts in ((1 / 3, 1 / 3, 1 / 3), (0.6, 0.3, 0.1), (0.15, 0.15, 0.7)):
        p = np.array(wts) @ tv
        d2, d3 = tri_derivs((p[0], p[1], 0.0), tv)
        f2, f3 = _polar_finite_parts(p, tv)
        sc2 = np.abs(f2).max()
        assert np.abs(d2[:2, :2] - f2[:2, :2]).max() <= 1e-11 * sc2
        assert abs(d2[2, 2] - f2[2, 2]) <= 1e-11 * sc2
        assert np.abs(d2[:2, 2]).max() <= 1e-14 * sc2  # odd in x3
        sc3 = np.abs(f3).max()
        assert np.abs(d3[:2, :2, :2] - f3[:2, :2, :2]).max() <= 1e-11 * sc3
        assert np.abs(d3[:2, :2, 2]).max() <= 1e-14 * sc3


def _brute_force(x, tv, n=48):
    """Collapsed Gauss rule on the triangle: xi = A + u (B - A) + u v (C - B), jacobian
    2 area u; the integrand the second and third x-derivatives of 1/R."""
    A, B, C = (np.array(v, dtype=float) for v in tv)
    area = 0.5 * abs((B - A)[0] * (C - A)[1] - (B - A)[1] * (C - A)[0])
    xg, wg = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (xg + 1)
    wu = 0.5 * wg
    U, Vv = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu) * 2 * area * U
    P = A + U[..., None] * (B - A) + (U * Vv)[..., None] * (C - B)
    d = np.stack([x[0] - P[..., 0], x[1] - P[..., 1], np.full(U.shape, x[2])], -1)
    R2 = (d * d).sum(-1)
    R = np.sqrt(R2)
    d2 = np.zeros((3, 3))
    d3 = np.zeros((3, 3, 3))
    for i, j in itertools.product(range(3), repeat=2):
        d2[i, j] = (W * (3 * d[..., i] * d[..., j] / R ** 5 - (i == j) / R ** 3)).sum()
        for k in range(3):
            dl = (i == j) * d[..., k] + (i == k) * d[..., j] + (j == k) * d[..., i]
            d3[i, j, k] = (W * (3 * dl / R ** 5 - 15 * d[..., i] * d[..., j] * d[..., k] / R ** 7)).sum()
    return d2, d3


@pytest.mark.parametrize("tv", [
    [(-0.4, -0.1), (0.5, -0.3), (0.1, 0.6)],
    [(0.0, 0.0), (2.0, 0.1), (0.3, 0.25)],
])
def test_off_plane_values_match_brute_force_quadrature(tv):
    rng = np.random.default_rng(3)
    for _ in range(6):
        x = np.array([*rng.uniform(-0.5, 1.0, 2), rng.choice([-1, 1]) * rng.uniform(0.6, 1.5)])
        d2, d3 = tri_derivs(x, tv)
        b2, b3 = _brute_force(x, tv)
        assert np.abs(d2 - b2).max() <= 1e-11 * np.abs(b2).max()
        assert np.abs(d3 - b3).max() <= 1e-11 * np.abs(b3).max()


def test_far_field_is_area_times_point_source():
    tv = np.array([(-0.4, -0.1), (0.5, -0.3), (0.1, 0.6)])
    c = tv.mean(axis=0)
    area = 0.5 * abs((tv[1] - tv[0])[0] * (tv[2] - tv[0])[1] - (tv[1] - tv[0])[1] * (tv[2] - tv[0])[0])
    for dist in (20.0, 80.0):
        x = np.array([c[0] + 0.6 * dist, c[1] - 0.3 * dist, 0.74 * dist])
        d2, _ = tri_derivs(x, tv)
        d = x - np.array([c[0], c[1], 0.0])
        r = np.linalg.norm(d)
        ref = area * (3 * np.outer(d, d) / r ** 5 - np.eye(3) / r ** 3)
        # the first moment about the centroid vanishes: error O((size / r)^2)
        assert np.abs(d2 - ref).max() <= 4.0 / r ** 2 * np.abs(ref).max()


def test_point_on_an_edge_is_singular():
    tv = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]
    assert O.tri_phi_derivatives((0.5, 0.0, 0.0), tv)[0] != 0
    assert O.tri_phi_derivatives((0.5, 0.5, 0.0), tv)[0] != 0
    assert O.tri_phi_derivatives((0.5, 0.0, 1e-3), tv)[0] == 0


def _tri_penny_error(n):
    el = synth.tri_disk_mesh(n)
    A = O.dense_matrix(el, E, NU)
    b = np.zeros((el.N, 3))
    b[:, 2] = -1.0
    x = np.linalg.solve(A, b.ravel()).reshape(-1, 3)
    r = np.linalg.norm(el.c, axis=1)
    exact = O.sneddon_opening(r, E, NU)
    return np.linalg.norm(x[:, 2] - exact) / np.linalg.norm(exact), x


def test_sneddon_penny_with_triangles():
    errs = [_tri_penny_error(n)[0] for n in (8, 16)]
    assert errs[1] < errs[0] < 0.2
    _, x = _tri_penny_error(16)
    assert np.all(x[:, 2] > 0)
