"""Pins of the oracle's cluster tree, block partition, tangent operator and GMRES (CPU).

Facts checked: the permutation is a bijection; leaves hold at most leaf_size
elements; every split is a median split along the longest centroid-box axis; the
near and far blocks tile the (N x N) element index square exactly once (brute-force
coverage count); every far block satisfies the admissibility inequality on boxes
recomputed from the element vertices; GMRES agrees with a direct LU solve and its
residual, recomputed independently, meets the tolerance; with the exact inverse as
preconditioner GMRES converges in one iteration.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import synth

E, NU = 1.0, 0.25


@pytest.fixture(scope="module")
def penny():
    el = synth.config_penny(40)
    return el, O.dense_matrix(el, E, NU)


@pytest.mark.parametrize("leaf", [16, 64])
def test_tree_is_a_bijection_with_bounded_leaves(leaf):
    el = synth.config_three_planes(12)
    T = O.cluster_tree(el, leaf)
    assert sorted(T.perm.tolist()) == list(range(el.N))
    for q in range(T.n_nodes):
        n = T.end[q] - T.begin[q]
        if T.is_leaf(q):
            assert 1 <= n <= leaf
        else:
            l, r = T.left[q], T.right[q]
            assert T.begin[l] == T.begin[q] and T.end[l] == T.begin[r] and T.end[r] == T.end[q]
            assert T.end[l] - T.begin[l] == n // 2
            # median split along the longest axis of the centroid box
            cc = el.c[T.perm[T.begin[q]:T.end[q]]]
            ax = int(np.argmax(cc.max(0) - cc.min(0)))
            cl = el.c[T.perm[T.begin[l]:T.end[l]], ax]
            cr = el.c[T.perm[T.begin[r]:T.end[r]], ax]
            assert cl.max() <= cr.min()


def test_blocks_tile_the_index_square_exactly_once():
    el = synth.config_three_planes(10)
    T = O.cluster_tree(el, 16)
    near, far = O.block_partition(T, 2.0)
    cover = np.zeros((el.N, el.N), dtype=np.int32)
    for s, t in near + far:
        rs = T.perm[T.begin[s]:T.end[s]]
        rt = T.perm[T.begin[t]:T.end[t]]
        cover[np.ix_(rs, rt)] += 1
    assert cover.min() == 1 and cover.max() == 1
    for s, t in near:
        assert T.is_leaf(s) and T.is_leaf(t)
    assert len(far) > 0


def test_far_blocks_are_admissible_on_vertex_boxes():
    el = synth.config_fault(48)
    T = O.cluster_tree(el, 32)
    near, far = O.block_partition(T, 2.0)
    # recompute the boxes from the explicit vertex list
    verts = []
    for sa in (-1, 1):
        for sb in (-1, 1):
            verts.append(el.c + sa * el.a[:, None] * el.s1 + sb * el.b[:, None] * el.s2)
    verts = np.stack(verts, 1)  # (N, 4, 3)

    def box(q):
        v = verts[T.perm[T.begin[q]:T.end[q]]].reshape(-1, 3)
        return v.min(0), v.max(0)

    for s, t in far:
        (ls, hs), (lt, ht) = box(s), box(t)
        ds, dt = np.linalg.norm(hs - ls), np.linalg.norm(ht - lt)
        gap = np.maximum(0.0, np.maximum(lt - hs, ls - ht))
        dist = np.linalg.norm(gap)
        assert dist > 0 and min(ds, dt) <= 2.0 * dist * (1 + 1e-12)
    # near leaf pairs of one plane touch or are close: none is admissible
    for s, t in near[:200]:
        assert not O.admissible(T, s, t, 2.0)


def test_gmres_matches_lu_on_the_penny_crack(penny):
    el, A = penny
    b = synth.rhs_uniform_pressure(el)
    x_lu = np.linalg.solve(A, b)
    x, its, ok, hist = O.gmres(lambda v: A @ v, b, tol=1e-10, restart=50)
    assert ok
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001
    assert np.linalg.norm(x - x_lu) <= 1e-8 * np.linalg.norm(x_lu)


def test_gmres_with_block_jacobi_and_stiffness(penny):
    el, E_ = penny
    rng = np.random.default_rng(3)
    h = 2.0 / 40
    k = np.exp(rng.uniform(math.log(1e-3), math.log(1e2), size=el.N)) * (E / h)
    A = O.tangent_dense(E_, k)
    assert np.allclose(np.diag(A), np.diag(E_) - np.repeat(k, 3))
    T = O.cluster_tree(el, 64)
    inv = O.block_jacobi_inverses(A, T)
    b = synth.rhs_normal(3 * el.N, 7)
    x0, its0, ok0, _ = O.gmres(lambda v: A @ v, b, tol=1e-8, restart=50)
    x1, its1, ok1, _ = O.gmres(lambda v: A @ v, b, lambda r: O.apply_block_jacobi(inv, r), tol=1e-8)
    assert ok0 and ok1 and its1 < its0
    ref = np.linalg.solve(A, b)
    for x in (x0, x1):
        assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
        assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)


def test_gmres_with_exact_preconditioner_takes_one_iteration(penny):
    el, A = penny
    Ainv = np.linalg.inv(A)
    b = synth.rhs_normal(3 * el.N, 9)
    x, its, ok, _ = O.gmres(lambda v: A @ v, b, lambda r: Ainv @ r, tol=1e-10)
    assert ok and its == 1


def test_gmres_restart_path():
    rng = np.random.default_rng(5)
    n = 200
    A = np.eye(n) * 3 + rng.normal(size=(n, n)) / math.sqrt(n)
    b = rng.normal(size=n)
    x, its, ok, _ = O.gmres(lambda v: A @ v, b, tol=1e-12, restart=5, maxit=500)
    assert ok and its > 5
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b) * 1.0001


def test_point_jacobi_is_block_jacobi_on_one_element_leaves(penny):
    """The 3x3 point Jacobi of every element equals leaf block-Jacobi on a tree whose
    leaves hold one element each; on a matrix that is block diagonal with 3x3 blocks it
    is the exact inverse (one GMRES iteration)."""
    el, E_ = penny
    rng = np.random.default_rng(4)
    k = np.exp(rng.uniform(math.log(1e-3), math.log(1e2), size=el.N)) * (E / (2.0 / 40))
    A = O.tangent_dense(E_, k, 0.1)
    pj = O.point_jacobi_inverses(A)
    bj = O.block_jacobi_inverses(A, O.cluster_tree(el, 1))
    r = rng.normal(size=3 * el.N)
    z1, z2 = O.apply_block_jacobi(pj, r), O.apply_block_jacobi(bj, r)
    assert np.abs(z1 - z2).max() <= 1e-12 * np.abs(z1).max()
    # each block applied separately: B_e z_e = r_e
    for e in rng.choice(el.N, size=20, replace=False):
        d = slice(3 * e, 3 * e + 3)
        assert np.allclose(A[d, d] @ z1[d], r[d], rtol=1e-12, atol=1e-12 * np.abs(r[d]).max())
    D = np.zeros_like(A)
    for e in range(el.N):
        D[3 * e:3 * e + 3, 3 * e:3 * e + 3] = A[3 * e:3 * e + 3, 3 * e:3 * e + 3]
    b = synth.rhs_normal(3 * el.N, 10)
    x, its, ok, _ = O.gmres(lambda v: D @ v, b, lambda q: O.apply_block_jacobi(pj, q), tol=1e-10)
    assert ok and its == 1
    # on the tangent: between no preconditioner and leaf block-Jacobi
    T = O.cluster_tree(el, 64)
    its_none = O.gmres(lambda v: A @ v, b, tol=1e-8)[1]
    its_pj = O.gmres(lambda v: A @ v, b, lambda q: O.apply_block_jacobi(pj, q), tol=1e-8)[1]
    its_bj = O.gmres(lambda v: A @ v, b, lambda q: O.apply_block_jacobi(O.block_jacobi_inverses(A, T), q),
                     tol=1e-8)[1]
    assert its_bj <= its_pj < its_none


def test_bicgstab_matches_lu_and_gmres(penny):
    """BiCGSTAB (the paper's A11 Krylov method) on the tangent: meets the tolerance on
    the recomputed residual and matches the LU solution, with and without block-Jacobi."""
    el, E_ = penny
    rng = np.random.default_rng(13)
    k = np.exp(rng.uniform(math.log(1e-3), math.log(1e2), size=el.N)) * (E / (2.0 / 40))
    A = O.tangent_dense(E_, k)
    inv = O.block_jacobi_inverses(A, O.cluster_tree(el, 64))
    b = synth.rhs_normal(3 * el.N, 14)
    ref = np.linalg.solve(A, b)
    for M in (None, lambda r: O.apply_block_jacobi(inv, r)):
        x, its, ok = O.bicgstab(lambda v: A @ v, b, M, tol=1e-10)
        assert ok and its > 0
        assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)


def test_bicgstab_finite_termination():
    """With the exact inverse as preconditioner one iteration solves the system; on
    I + u v^T (a Krylov space of dimension 2) BiCGSTAB ends within two iterations; a
    nonsymmetric system with a known solution is solved to the tolerance."""
    rng = np.random.default_rng(15)
    n = 60
    A = np.eye(n) * 2 + rng.normal(size=(n, n)) / math.sqrt(n)
    b = rng.normal(size=n)
    Ainv = np.linalg.inv(A)
    x, its, ok = O.bicgstab(lambda v: A @ v, b, lambda r: Ainv @ r, tol=1e-12)
    assert ok and its == 1 and np.allclose(x, Ainv @ b, rtol=1e-12, atol=1e-12)
    u, v = rng.normal(size=n), rng.normal(size=n) * 0.1
    B = np.eye(n) + np.outer(u, v)
    x, its, ok = O.bicgstab(lambda w: B @ w, b, tol=1e-12)
    assert ok and its <= 2
    assert np.linalg.norm(B @ x - b) <= 1e-12 * np.linalg.norm(b)
    xs = rng.normal(size=n)
    x, its, ok = O.bicgstab(lambda w: A @ w, A @ xs, tol=1e-13)
    assert ok and np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
