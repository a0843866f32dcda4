"""Pins of the flow and coupled-Jacobian oracle (oracle/flow.py; Sec. 3.2, 3.3, 3.3.1)
against what the finite-element method and linear algebra fix:

* the element matrices equal the closed forms of the bilinear rectangle, written out
  here: mass A/36 [[4,2,1,2],...], stiffness (b/a)/6 Kx + (a/b)/6 Ky, load A/4 per node;
* the stiffness annihilates constants and, on a uniform grid, a linear pressure field
  leaves no residual at interior nodes (patch test); the mass matrix integrates 1 to the
  area;
* N_p returns the centroid value of a bilinear field;
* A21 and A22 equal central differences of the flow residual (the exact Jacobian);
* with the exact Schur complement, GMRES right-preconditioned by P_up converges in at
  most two iterations (a block-triangular preconditioner with the exact Schur
  complement has a minimal polynomial of degree two).
"""
import numpy as np
import pytest

from oracle import flow as F
from oracle import oracle as O
from paper_2605_14397_gb300 import synth

KX = np.array([[2, -2, -1, 1], [-2, 2, 1, -1], [-1, 1, 2, -2], [1, -1, -2, 2]], dtype=float)
KY = np.array([[2, 1, -1, -2], [1, 2, -2, -1], [-1, -2, 2, 1], [-2, -1, 1, 2]], dtype=float)
MASS = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]], dtype=float)


@pytest.mark.parametrize("a,b", [(0.5, 0.5), (0.3, 0.7), (2.0, 0.1)])
def test_element_matrices_closed_form(a, b):
    m, k, v = F.element_matrices(a, b)
    A = 4 * a * b
    assert np.allclose(m, A / 36 * MASS, rtol=1e-14, atol=0)
    assert np.allclose(k, (b / a) / 6 * KX + (a / b) / 6 * KY, rtol=1e-14, atol=1e-15)
    assert np.allclose(v, np.full(4, A / 4), rtol=1e-14, atol=0)
    assert abs(m.sum() - A) <= 1e-14 * A
    assert np.abs(k @ np.ones(4)).max() <= 1e-14 * np.abs(k).max()


def node_xy(el, conn, n_nodes):
    """In-plane coordinates of the nodes of a single plane (s1, s2 of element 0)."""
    sg = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=float)
    xy = np.zeros((n_nodes, 2))
    for e in range(el.N):
        c = np.array([el.c[e] @ el.s1[0], el.c[e] @ el.s2[0]])
        for i in range(4):
            xy[conn[e, i]] = c + sg[i] * [el.a[e], el.b[e]]
    return xy


def test_patch_test_and_centroid_interpolation():
    el = synth.plane_grid(5, 4, -1.0, 1.0, -0.6, 0.6, (0, 0, 1))
    conn, nn = synth.node_connectivity(el)
    xy = node_xy(el, conn, nn)
    V, S, L = F.assemble(conn, nn, el.a, el.b, np.zeros(el.N), M=2.0, mu=0.5, w0=1.0)
    p = 0.3 + 1.7 * xy[:, 0] - 0.9 * xy[:, 1]
    r = L @ p
    edge = (np.isclose(np.abs(xy[:, 0]), 1.0)) | (np.isclose(np.abs(xy[:, 1]), 0.6))
    assert np.abs(r[~edge]).max() <= 1e-13 and np.abs(r[edge]).max() > 1e-3
    assert abs(S.sum() - 2.0 * 1.2 / 2.0) <= 1e-13       # w / M times the area
    assert abs(V.sum() - 2.0 * 1.2) <= 1e-13
    A12, _, _ = F.jacobian_blocks(conn, nn, el.a, el.b, np.zeros(el.N), np.zeros(nn), np.zeros(nn),
                                  M=2.0, mu=0.5, w0=1.0, dt=0.1)
    q = 0.2 - xy[:, 0] + 0.4 * xy[:, 1] + 0.7 * xy[:, 0] * xy[:, 1]   # bilinear field
    cx = el.c @ el.s1[0]
    cy = el.c @ el.s2[0]
    pc = (A12 @ q)[2::3]
    assert np.allclose(pc, 0.2 - cx + 0.4 * cy + 0.7 * cx * cy, rtol=0, atol=1e-14)
    assert np.all((A12 @ q)[0::3] == 0) and np.all((A12 @ q)[1::3] == 0)


def test_jacobian_is_the_derivative_of_the_residual():
    el = synth.config_three_planes(4)
    conn, nn = synth.node_connectivity(el)
    rng = np.random.default_rng(3)
    par = dict(M=3.0, mu=0.7, w0=0.05, dt=0.2)
    dn_old = rng.uniform(0.0, 0.05, el.N)
    ddn = rng.uniform(-0.01, 0.02, el.N)
    dp = rng.normal(size=nn)
    pn = rng.normal(size=nn)
    f = rng.normal(size=nn)
    A12, A21, A22 = F.jacobian_blocks(conn, nn, el.a, el.b, dn_old + ddn, dp, pn, par["M"], par["mu"], par["w0"],
                                      par["dt"])

    def rf(ddn_, dp_):
        return F.flow_residual(conn, nn, el.a, el.b, dn_old, ddn_, dp_, pn, f, par["M"], par["mu"], par["w0"],
                               par["dt"])
    h = 1e-6
    for e in range(0, el.N, 7):
        d = np.zeros(el.N)
        d[e] = h
        col = (rf(ddn + d, dp) - rf(ddn - d, dp)) / (2 * h)
        assert np.abs(col - A21[:, 3 * e + 2]).max() <= 1e-7 * max(1.0, np.abs(col).max())
        assert np.all(A21[:, 3 * e] == 0) and np.all(A21[:, 3 * e + 1] == 0)
    for j in range(0, nn, 9):
        d = np.zeros(nn)
        d[j] = h
        col = (rf(ddn, dp + d) - rf(ddn, dp - d)) / (2 * h)
        assert np.abs(col - A22[:, j]).max() <= 1e-7 * max(1.0, np.abs(col).max())


def test_exact_schur_complement_gives_two_iterations():
    el = synth.config_three_planes(4)
    conn, nn = synth.node_connectivity(el)
    Em = O.dense_matrix(el, 1.0, 0.25)
    rng = np.random.default_rng(4)
    A11 = O.tangent_dense(Em, rng.uniform(1.0, 5.0, el.N), 0.1)
    A12, A21, A22 = F.jacobian_blocks(conn, nn, el.a, el.b, rng.uniform(0, 0.05, el.N), rng.normal(size=nn),
                                      rng.normal(size=nn), M=3.0, mu=0.7, w0=0.05, dt=0.2)
    J = F.coupled(A11, A12, A21, A22)
    n1 = 3 * el.N
    b = rng.normal(size=J.shape[0])
    S_exact = A22 - A21 @ np.linalg.solve(A11, A12)
    x, its, ok, _ = O.gmres(lambda v: J @ v, b, lambda y: F.apply_pup_inverse(A11, A12, S_exact, y, n1), tol=1e-10)
    assert ok and its <= 2
    x2, its2, ok2, _ = O.gmres(lambda v: J @ v, b,
                               lambda y: F.apply_pup_inverse(A11, A12, F.schur_diag(A11, A12, A21, A22), y, n1),
                               tol=1e-10)
    assert ok2 and its2 > its
    assert np.allclose(x, np.linalg.solve(J, b), rtol=1e-8, atol=1e-10)


# ------------------------------------------------------------------ linear triangles

def _cot(u, v):
    return float(np.dot(u, v) / np.linalg.norm(np.cross(u, v)))


@pytest.mark.parametrize("V", [
    [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)],
    [(0.1, -0.2, 0.3), (0.9, 0.1, 0.2), (0.2, 0.7, -0.4)],   # oblique, in 3D
    [(0.0, 0.0, 0.0), (2.0, 0.1, 0.0), (0.3, 0.25, 0.0)],    # obtuse
])
def test_triangle_element_matrices_closed_forms(V):
    """Mass A/12 (1 + delta_ij), load A/3, stiffness by the cotangent formula
    k_ij = -cot(theta_k) / 2 (theta_k the angle at the third vertex), rows summing to 0."""
    V = np.array(V)
    m, k, v = F.tri_element_matrices(V)
    A = 0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
    assert np.allclose(m, A / 12 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-13, atol=0)
    assert np.allclose(v, np.full(3, A / 3), rtol=1e-13, atol=0)
    ref = np.zeros((3, 3))
    for i in range(3):
        j, l = (i + 1) % 3, (i + 2) % 3
        th = _cot(V[i] - V[l], V[j] - V[l])  # angle at l, opposite the edge (i, j)
        ref[i, j] = ref[j, i] = -0.5 * th
    for i in range(3):
        ref[i, i] = -ref[i].sum()
    assert np.abs(k - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(k @ np.ones(3)).max() <= 1e-13 * np.abs(k).max()


def test_triangle_patch_test_and_centroid_interpolation():
    """On a jittered triangulation a linear pressure leaves no residual L p at interior
    nodes (P1 reproduces linear fields), and N_p returns its centroid value."""
    el = synth.tri_disk_mesh(8, jitter=0.2, seed=5)
    conn, nn = synth.node_connectivity(el)
    assert np.all(conn[:, 3] == -1)
    xyz = np.zeros((nn, 3))
    for e in range(el.N):
        xyz[conn[e, :3]] = el.tri[e].reshape(3, 3)
    V, S, L = F.assemble(conn, nn, el.a, el.b, np.zeros(el.N), M=2.0, mu=0.5, w0=1.0, shape=el.shape, tri=el.tri)
    p = 0.3 + 1.7 * xyz[:, 0] - 0.9 * xyz[:, 1]
    r = L @ p
    # interior nodes: the angles of their triangles sum to 2 pi
    ang = np.zeros(nn)
    for e in range(el.N):
        P = el.tri[e].reshape(3, 3)
        for i in range(3):
            u, w = P[(i + 1) % 3] - P[i], P[(i + 2) % 3] - P[i]
            ang[conn[e, i]] += np.arccos(np.dot(u, w) / np.linalg.norm(u) / np.linalg.norm(w))
    interior = np.abs(ang - 2 * np.pi) < 1e-9
    assert interior.sum() > 10
    assert np.abs(r[interior]).max() <= 1e-12 * np.abs(r).max()
    area = 0.5 * np.linalg.norm(np.cross(el.tri[:, 3:6] - el.tri[:, 0:3], el.tri[:, 6:9] - el.tri[:, 0:3]), axis=1)
    assert abs(V.sum() - area.sum()) <= 1e-13 * area.sum()
    A12, _, _ = F.jacobian_blocks(conn, nn, el.a, el.b, np.zeros(el.N), np.zeros(nn), np.zeros(nn),
                                  M=2.0, mu=0.5, w0=1.0, dt=0.1, shape=el.shape, tri=el.tri)
    pc = (A12 @ p)[2::3]
    assert np.allclose(pc, 0.3 + 1.7 * el.c[:, 0] - 0.9 * el.c[:, 1], rtol=0, atol=1e-13)


def _mixed_flow_mesh():
    """Triangles and rectangles sharing nodes: a rectangular grid whose left half is
    split into triangles (the same vertices)."""
    el = synth.plane_grid(6, 4, -0.3, 0.3, -0.2, 0.2, (0, 0, 1))
    parts, tris = [], []
    for e in range(el.N):
        c, a, b = el.c[e], el.a[e], el.b[e]
        s1, s2 = el.s1[e], el.s2[e]
        P = [c - a * s1 - b * s2, c + a * s1 - b * s2, c + a * s1 + b * s2, c - a * s1 + b * s2]
        if c[0] < 0:
            tris += [(P[0], P[1], P[2]), (P[0], P[2], P[3])]
        else:
            parts.append(el.subset([e]))
    return synth.Elements.concat([synth.triangles(np.array(tris), (0, 0, 1))] + parts)


def test_mixed_mesh_jacobian_is_the_derivative_of_the_residual():
    el = _mixed_flow_mesh()
    conn, nn = synth.node_connectivity(el)
    assert (el.shape == 1).sum() == 24 and (el.shape == 0).sum() == 12
    # the two shapes share the nodes of their common edge
    tri_nodes = set(conn[el.shape == 1][:, :3].ravel())
    rect_nodes = set(conn[el.shape == 0].ravel())
    assert len(tri_nodes & rect_nodes) == 5
    rng = np.random.default_rng(6)
    par = dict(M=3.0, mu=0.7, w0=0.05, dt=0.2)
    dn_old = rng.uniform(0.0, 0.05, el.N)
    ddn = rng.uniform(-0.01, 0.02, el.N)
    dp = rng.normal(size=nn)
    pn = rng.normal(size=nn)
    f = rng.normal(size=nn)
    kw = dict(shape=el.shape, tri=el.tri)
    A12, A21, A22 = F.jacobian_blocks(conn, nn, el.a, el.b, dn_old + ddn, dp, pn, par["M"], par["mu"], par["w0"],
                                      par["dt"], **kw)

    def rf(ddn_, dp_):
        return F.flow_residual(conn, nn, el.a, el.b, dn_old, ddn_, dp_, pn, f, par["M"], par["mu"], par["w0"],
                               par["dt"], **kw)
    h = 1e-6
    for e in range(0, el.N, 3):
        d = np.zeros(el.N)
        d[e] = h
        col = (rf(ddn + d, dp) - rf(ddn - d, dp)) / (2 * h)
        assert np.abs(col - A21[:, 3 * e + 2]).max() <= 1e-7 * max(1.0, np.abs(col).max())
    for j in range(0, nn, 4):
        d = np.zeros(nn)
        d[j] = h
        col = (rf(ddn, dp + d) - rf(ddn, dp - d)) / (2 * h)
        assert np.abs(col - A22[:, j]).max() <= 1e-7 * max(1.0, np.abs(col).max())
    # N_p: 1/3 on a triangle's nodes, 1/4 on a rectangle's
    rows = A12[2::3]
    assert np.allclose(rows[el.shape == 1].sum(axis=1), 1.0) and np.allclose(rows[el.shape == 1].max(axis=1), 1 / 3)
    assert np.allclose(rows[el.shape == 0].max(axis=1), 0.25)
