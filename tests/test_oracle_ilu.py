"""Pins of the oracle's sparse tangent approximation and ILU(0) preconditioner
(oracle/ilu.py, Sec. 3.3.1) against what the mathematics fixes: on a full pattern ILU(0)
is the exact LU factorization, on a tridiagonal matrix (no fill) too; on any pattern
(L U)_ab = A_ab at every entry of the pattern while the fill outside it is dropped; the
selection of the largest near-field entries against brute force, ties included; the
near-field entries against the dense E block by block; with every block near and p = 1
the sparse approximation is the tangent itself and preconditioned GMRES takes one
iteration, in either factorization order.  The leaf-colour order: a proper colouring
within the greedy bound, a permutation grouped by colour and leaf, a solve no deeper
than the colours times the deepest single leaf."""
import math

import numpy as np
import pytest

from oracle import ilu as IL
from oracle import oracle as O
from paper_2605_14397_gb300 import synth

E, NU = 1.0, 0.25


def rows_of(M, pattern=None):
    n = M.shape[0]
    if pattern is None:
        pattern = np.ones_like(M, dtype=bool)
    return [{b: M[a, b] for b in range(n) if pattern[a, b]} for a in range(n)]


def lu_product(L, U):
    n = len(L)
    Ld = np.eye(n)
    for a, r in enumerate(L):
        for b, x in r.items():
            Ld[a, b] = x
    return Ld @ IL.to_dense(U)


def diag_dominant(n, rng, pattern=None):
    M = rng.normal(size=(n, n))
    if pattern is not None:
        M = np.where(pattern, M, 0.0)
    M[np.arange(n), np.arange(n)] = np.abs(M).sum(axis=1) + 1.0
    return M


def test_full_pattern_is_exact_lu():
    rng = np.random.default_rng(0)
    A = diag_dominant(12, rng)
    L, U = IL.ilu0(rows_of(A))
    assert np.allclose(lu_product(L, U), A, rtol=0, atol=1e-12 * np.abs(A).max())
    r = rng.normal(size=12)
    assert np.allclose(IL.ilu0_solve(L, U, r), np.linalg.solve(A, r), rtol=1e-12, atol=1e-14)


def test_tridiagonal_has_no_fill():
    rng = np.random.default_rng(1)
    n = 30
    pat = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 1
    A = diag_dominant(n, rng, pat)
    L, U = IL.ilu0(rows_of(A, pat))
    r = rng.normal(size=n)
    assert np.allclose(IL.ilu0_solve(L, U, r), np.linalg.solve(A, r), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_product_matches_on_the_pattern_and_drops_fill(seed):
    rng = np.random.default_rng(seed)
    n = 25
    pat = rng.random((n, n)) < 0.2
    pat[np.arange(n), np.arange(n)] = True
    A = diag_dominant(n, rng, pat)
    L, U = IL.ilu0(rows_of(A, pat))
    for a in range(n):
        assert all(b < a and pat[a, b] for b in L[a])
        assert all(b >= a and pat[a, b] for b in U[a])
    P = lu_product(L, U)
    assert np.allclose(P[pat], A[pat], rtol=0, atol=1e-12 * np.abs(A).max())
    # this pattern has fill: the dropped products are not zero, so L U differs from A off it
    assert np.abs(P[~pat]).max() > 1e-6


def test_selection_against_brute_force_with_ties():
    rng = np.random.default_rng(5)
    n = 400
    i = rng.integers(0, 50, size=n)
    j = rng.integers(0, 50, size=n)
    v = rng.choice([-3.0, -2.0, 1.0, 2.0, 3.0, 0.5], size=n)  # many equal magnitudes
    for p in (0.01, 0.1, 0.37, 1.0):
        si, sj, sv = IL.select_largest(i, j, v, p)
        m = int(math.ceil(p * n))
        assert sv.size == m
        key = sorted(range(n), key=lambda q: (-abs(v[q]), i[q], j[q]))[:m]
        assert list(zip(si, sj, sv)) == [(i[q], j[q], v[q]) for q in key]
    with pytest.raises(ValueError):
        IL.select_largest(i, j, v, 0.0)


def test_near_entries_are_the_near_blocks_of_E():
    el = synth.config_three_planes(6)  # not symmetric: a transposed block would show
    Em = O.dense_matrix(el, E, NU)
    assert np.abs(Em - Em.T).max() > 1e-3 * np.abs(Em).max()
    T = O.cluster_tree(el, 8)
    i, j, v = IL.near_entries(Em, T)
    near, _ = O.block_partition(T, 2.0)
    sizes = [(T.end[s] - T.begin[s]) * (T.end[t] - T.begin[t]) for s, t in near]
    assert v.size == 9 * sum(sizes)
    cd = IL.cluster_dofs(T)
    assert np.array_equal(v, Em[cd[i], cd[j]])
    assert len(set(zip(i.tolist(), j.tolist()))) == v.size  # no entry twice
    diag = set(np.nonzero(i == j)[0].tolist())
    assert len(diag) == Em.shape[0]  # the self blocks are near


def test_all_near_and_p_one_gives_the_tangent():
    el = synth.config_penny(8)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    eta = 1e-12  # nothing admissible: every leaf pair is near
    k = synth.k_loguniform(el.N, 7, h=0.25)
    A = O.tangent_dense(Em, k, shift=0.3)
    rows = IL.sparse_tangent(Em, T, k, p=1.0, eta=eta, shift=0.3)
    cd = IL.cluster_dofs(T)
    assert np.array_equal(IL.to_dense(rows), A[np.ix_(cd, cd)])
    M, nnz = IL.ilu_preconditioner(Em, T, k, p=1.0, eta=eta, shift=0.3)
    assert nnz == A.size
    b = synth.rhs_normal(A.shape[0], 8)
    x, its, conv, _ = O.gmres(lambda u: A @ u, b, M, tol=1e-10)
    assert conv and its == 1
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def interface_blocks(N, seed):
    """Seeded 3x3 tangent blocks: the oracle's consistent tangents of seeded interface
    states (Sec. 2.2), a mix of elastic, Coulomb and apex returns."""
    from oracle import interface as IF
    P = IF.Params(**synth.INTERFACE_PARAMS["softening"])
    T, dp, chi, dd = synth.interface_states(N, seed)
    return IF.step_all(P, T, dp, chi, dd)[4]


def test_cep_blocks_reduce_to_the_diagonal_path():
    el = synth.config_penny(6)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    k = synth.k_loguniform(el.N, 5, h=1 / 3)
    cep = np.zeros((el.N, 3, 3))
    cep[:, [0, 1, 2], [0, 1, 2]] = k[:, None]
    # the same values up to the order of the two subtractions
    tol = 4e-16 * np.abs(O.tangent_dense(Em, k, 0.2)).max()
    assert np.abs(O.tangent_dense(Em, k, 0.2) - O.tangent_dense(Em, None, 0.2, cep=cep)).max() <= tol
    for p in (0.05, 1.0):
        a = IL.sparse_tangent(Em, T, k, p=p, shift=0.2)
        b = IL.sparse_tangent(Em, T, None, p=p, shift=0.2, cep=cep)
        for ra, rb in zip(a, b):        # b also holds the (zero) off-diagonal block entries
            assert all(abs(rb[c] - x) <= tol for c, x in ra.items())
            assert all(c in ra or x == 0.0 for c, x in rb.items())


def test_all_near_and_p_one_gives_the_tangent_with_cep():
    el = synth.config_penny(8)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    eta = 1e-12
    k = synth.k_loguniform(el.N, 7, h=0.25)
    cep = interface_blocks(el.N, 11)
    A = O.tangent_dense(Em, k, shift=0.3, cep=cep)
    # the blocks land on each element's own DOFs, off-diagonals included
    Ak = O.tangent_dense(Em, k, shift=0.3)
    e = 5
    assert np.array_equal(Ak[3 * e:3 * e + 3, 3 * e:3 * e + 3] - A[3 * e:3 * e + 3, 3 * e:3 * e + 3], cep[e])
    rows = IL.sparse_tangent(Em, T, k, p=1.0, eta=eta, shift=0.3, cep=cep)
    cd = IL.cluster_dofs(T)
    assert np.allclose(IL.to_dense(rows), A[np.ix_(cd, cd)], rtol=0, atol=1e-15 * np.abs(A).max())
    M, nnz = IL.ilu_preconditioner(Em, T, k, p=1.0, eta=eta, shift=0.3, cep=cep)
    b = synth.rhs_normal(A.shape[0], 8)
    x, its, conv, _ = O.gmres(lambda u: A @ u, b, M, tol=1e-10)
    assert conv and its == 1


def test_cep_pattern_holds_every_element_block():
    el = synth.config_penny(10)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    cep = interface_blocks(el.N, 12)
    rows = IL.sparse_tangent(Em, T, None, p=0.01, cep=cep)
    for a in range(len(rows)):
        for c in range(3):
            assert 3 * (a // 3) + c in rows[a]


def test_pattern_keeps_the_diagonal_and_the_count():
    el = synth.config_penny(10)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    k = synth.k_loguniform(el.N, 9, h=0.2)
    i, j, v = IL.near_entries(Em, T)
    for p in (0.001, 0.01, 0.05):
        rows = IL.sparse_tangent(Em, T, k, p=p)
        n = Em.shape[0]
        assert all(a in rows[a] for a in range(n))
        sel = set(zip(*IL.select_largest(i, j, v, p)[:2]))
        extra_diag = sum(1 for a in range(n) if (a, a) not in sel)
        assert sum(len(r) for r in rows) == int(math.ceil(p * v.size)) + extra_diag


def test_preconditioner_converges_on_a_tangent_system():
    """Empirical, not a pin: ILU(0) on the 5 % largest near-field entries cuts the
    unpreconditioned iteration count by more than ten on a penny crack with a
    log-uniform stiffness, and the preconditioned solve meets the tolerance."""
    el = synth.config_penny(16)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 16)
    k = synth.k_loguniform(el.N, 1605, h=2.0 / 16)
    A = O.tangent_dense(Em, k)
    b = synth.rhs_normal(A.shape[0], 3)
    _, its0, _, _ = O.gmres(lambda u: A @ u, b, None, tol=1e-8)
    M, _ = IL.ilu_preconditioner(Em, T, k, p=0.05)
    x, its, conv, _ = O.gmres(lambda u: A @ u, b, M, tol=1e-8)
    assert conv and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    assert 10 * its < its0


def _penny_rows(n=24, p=0.01, leaf=16):
    el = synth.config_penny(n)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, leaf)
    k = synth.k_loguniform(el.N, 1605, h=2.0 / n)
    return el, Em, T, k, IL.sparse_tangent(Em, T, k, p=p)


def test_leaf_colouring_is_proper_and_order_is_grouped():
    el, Em, T, k, rows = _penny_rows()
    leaf = IL.leaf_of_position(T)
    col = IL.leaf_colours(rows, T)
    deg = {}
    for a, r in enumerate(rows):
        for c in r:
            if leaf[c] != leaf[a]:
                assert col[leaf[c]] != col[leaf[a]]
                deg.setdefault(leaf[a], set()).add(leaf[c])
                deg.setdefault(leaf[c], set()).add(leaf[a])
    assert col.max() + 1 <= 1 + max(len(v) for v in deg.values())  # greedy bound
    order = IL.colour_order(rows, T)
    assert np.array_equal(np.sort(order), np.arange(len(rows)))
    cseq = col[leaf[order]]
    assert np.all(np.diff(cseq) >= 0)  # colour by colour
    lseq = leaf[order]
    starts = np.nonzero(np.diff(lseq))[0] + 1
    assert len(set(lseq[starts])) == len(starts)  # each leaf one contiguous run
    within = np.diff(order)[np.diff(lseq) == 0]
    assert np.all(within == 1)  # cluster order inside a leaf
    # leaves of one colour are not coupled, so the colour order's solve is no deeper
    # than the colours times the deepest single-leaf solve
    P = IL.permute_rows(rows, order)
    leaf_depth = max(IL.solve_depth([{c - lo: x for c, x in rows[a].items() if lo <= c < hi}
                                     for a in range(lo, hi)])
                     for lo, hi in [(3 * T.begin[q], 3 * T.end[q]) for q in T.leaves()])
    assert IL.solve_depth(P) <= (col.max() + 1) * leaf_depth


def test_colour_order_factorization_properties():
    el, Em, T, k, rows = _penny_rows()
    order = IL.colour_order(rows, T)
    P = IL.permute_rows(rows, order)
    L, U = IL.ilu0(P)
    A = IL.to_dense(P)
    pat = A != 0.0
    for a in range(len(P)):
        pat[a, list(P[a].keys())] = True
    assert np.allclose(lu_product(L, U)[pat], A[pat], rtol=0, atol=1e-12 * np.abs(A).max())
    # the permuted pattern is the original one renumbered
    assert sum(len(r) for r in P) == sum(len(r) for r in rows)


def test_colour_order_is_exact_when_everything_is_kept():
    el = synth.config_penny(8)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 8)
    k = synth.k_loguniform(el.N, 7, h=0.25)
    A = O.tangent_dense(Em, k)
    M, _ = IL.ilu_preconditioner(Em, T, k, p=1.0, eta=1e-12, ordering="colour")
    b = synth.rhs_normal(A.shape[0], 10)
    x, its, conv, _ = O.gmres(lambda u: A @ u, b, M, tol=1e-10)
    assert conv and its == 1
    with pytest.raises(ValueError):
        IL.ilu_preconditioner(Em, T, k, p=1.0, ordering="rcm")
