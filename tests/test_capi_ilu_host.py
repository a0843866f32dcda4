"""The library's host building blocks of the ILU preconditioner (hm_ilu_*, Sec. 3.3.1)
against the oracle (oracle/ilu.py), through the C-ABI, on CPU: the selection of the
largest near-field entries index for index, the CSR of the sparse tangent and its
ILU(0) bit for bit in both factorization orders, the levels of the triangular solves
against the oracle's depth and their defining recurrence, the leaf colouring colour for
colour; bad arguments return status codes."""
import ctypes

import numpy as np
import pytest

from oracle import ilu as IL
from oracle import oracle as O
from paper_2605_14397_gb300 import hmat, synth

E, NU = 1.0, 0.25


def to_csr(rows):
    rowptr = [0]
    col, val = [], []
    for r in rows:
        cs = sorted(r)
        col += cs
        val += [r[c] for c in cs]
        rowptr.append(len(col))
    return np.array(rowptr, np.int64), np.array(col, np.int32), np.array(val, np.float64)


def factored_rows(rowptr, col, lu, n):
    L = [{int(col[q]): lu[q] for q in range(rowptr[a], rowptr[a + 1]) if col[q] < a} for a in range(n)]
    U = [{int(col[q]): lu[q] for q in range(rowptr[a], rowptr[a + 1]) if col[q] >= a} for a in range(n)]
    return L, U


@pytest.fixture(scope="module")
def penny():
    el = synth.config_penny(20)
    Em = O.dense_matrix(el, E, NU)
    T = O.cluster_tree(el, 16)
    k = synth.k_loguniform(el.N, 1605, h=0.1)
    return el, Em, T, k


def test_selection_matches_oracle(penny):
    el, Em, T, k = penny
    i, j, v = IL.near_entries(Em, T)
    for p in (0.003, 0.01, 0.2, 1.0):
        got = hmat.ilu_select(i, j, v, p)
        order = np.lexsort((j, i, -np.abs(v)))[:int(np.ceil(p * v.size))]
        assert np.array_equal(got, order)
    # ties: many equal magnitudes, broken by (i, j)
    rng = np.random.default_rng(3)
    ti = rng.integers(0, 20, 300).astype(np.int32)
    tj = rng.integers(0, 20, 300).astype(np.int32)
    tv = rng.choice([1.0, -1.0, 2.0, -0.5], 300)
    si, sj, sv = IL.select_largest(ti, tj, tv, 0.3)
    got = hmat.ilu_select(ti, tj, tv, 0.3)
    assert np.array_equal(ti[got], si) and np.array_equal(tj[got], sj) and np.array_equal(tv[got], sv)


@pytest.mark.parametrize("ordering", ["cluster", "colour"])
@pytest.mark.parametrize("p", [0.01, 0.05])
def test_setup_chain_bit_identical_to_oracle(penny, ordering, p):
    """selection -> CSR assembly (with -k on the diagonal, renumbered) -> ILU(0), all in
    the library, against the oracle's sparse tangent and ILU(0)."""
    el, Em, T, k = penny
    shift = 0.25
    rows = IL.sparse_tangent(Em, T, k, p=p, shift=shift)
    i, j, v = IL.near_entries(Em, T)
    idx = hmat.ilu_select(i, j, v, p)
    d = np.repeat(k, 3)[IL.cluster_dofs(T)] + shift
    order = None
    if ordering == "colour":
        rp0, c0, _ = hmat.ilu_assemble(len(rows), idx, i, j, v, d)
        leaf = IL.leaf_of_position(T)
        colours, _ = hmat.ilu_leaf_colours(rp0, c0, leaf, int(leaf.max()) + 1)
        order = np.lexsort((np.arange(leaf.size), leaf, colours[leaf]))
        assert np.array_equal(order, IL.colour_order(rows, T))
        rows = IL.permute_rows(rows, order)
    rowptr, col, val = hmat.ilu_assemble(len(rows), idx, i, j, v, d, order)
    ro, co, vo = to_csr(rows)
    assert np.array_equal(rowptr, ro) and np.array_equal(col, co) and np.array_equal(val, vo)
    lu = hmat.ilu0_factor(rowptr, col, val)
    Lo, Uo = IL.ilu0(rows)
    L, U = factored_rows(rowptr, col, lu, len(rows))
    assert L == Lo and U == Uo  # same operations in the same order: equal bits


def test_levels_match_the_recurrence_and_the_oracle_depth(penny):
    el, Em, T, k = penny
    rows = IL.sparse_tangent(Em, T, k, p=0.05)
    rowptr, col, _ = to_csr(rows)
    lo, up, nl, nu = hmat.ilu_levels(rowptr, col)
    n = len(rows)
    for a in range(n):
        left = [lo[c] for c in rows[a] if c < a]
        right = [up[c] for c in rows[a] if c > a]
        assert lo[a] == (1 + max(left) if left else 0)
        assert up[a] == (1 + max(right) if right else 0)
    assert nl == IL.solve_depth(rows) and nl == lo.max() + 1 and nu == up.max() + 1
    # upper solve of the matrix = lower solve of the reversed matrix
    rev = [{n - 1 - c: x for c, x in rows[n - 1 - a].items()} for a in range(n)]
    assert nu == IL.solve_depth(rev)


def test_leaf_colours_match_oracle(penny):
    el, Em, T, k = penny
    rows = IL.sparse_tangent(Em, T, k, p=0.01)
    rowptr, col, _ = to_csr(rows)
    leaf = IL.leaf_of_position(T)
    nl = int(leaf.max()) + 1
    colours, nc = hmat.ilu_leaf_colours(rowptr, col, leaf, nl)
    ref = IL.leaf_colours(rows, T)
    assert np.array_equal(colours, ref) and nc == ref.max() + 1


def test_bad_arguments_return_status():
    rp = np.array([0, 1, 3], np.int64)
    col_ok = np.array([0, 0, 1], np.int32)
    with pytest.raises(hmat.HMError) as e:  # columns not increasing
        hmat.ilu0_factor(rp, np.array([0, 1, 0], np.int32), np.ones(3))
    assert e.value.status == hmat.HM_EINVAL
    with pytest.raises(hmat.HMError) as e:  # no diagonal in row 1
        hmat.ilu0_factor(np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), np.ones(2))
    assert e.value.status == hmat.HM_EINVAL
    with pytest.raises(hmat.HMError) as e:  # zero pivot
        hmat.ilu0_factor(rp, col_ok, np.array([0.0, 1.0, 1.0]))
    assert e.value.status == hmat.HM_EBREAKDOWN
    with pytest.raises(hmat.HMError) as e:
        hmat.ilu_select(np.zeros(3, np.int32), np.zeros(3, np.int32), np.ones(3), 0.0)
    assert e.value.status == hmat.HM_EINVAL
    with pytest.raises(hmat.HMError) as e:
        hmat.ilu_select(np.zeros(3, np.int32), np.zeros(3, np.int32), np.array([1.0, np.nan, 2.0]), 0.5)
    assert e.value.status == hmat.HM_ENAN
    with pytest.raises(hmat.HMError) as e:  # leaf out of range
        hmat.ilu_leaf_colours(rp, col_ok, np.array([0, 2], np.int32), 2)
    assert e.value.status == hmat.HM_EINVAL
    ii = np.array([0, 1, 1], np.int32)
    jj = np.array([1, 0, 0], np.int32)
    vv = np.ones(3)
    with pytest.raises(hmat.HMError) as e:  # the same position twice
        hmat.ilu_assemble(2, np.array([1, 2]), ii, jj, vv, np.zeros(2))
    assert e.value.status == hmat.HM_EINVAL
    with pytest.raises(hmat.HMError) as e:  # not a permutation
        hmat.ilu_assemble(2, np.array([0]), ii, jj, vv, np.zeros(2), order=np.array([1, 1]))
    assert e.value.status == hmat.HM_EINVAL
    rp2, c2, v2 = hmat.ilu_assemble(2, np.array([0, 1]), ii, jj, vv, np.array([3.0, 4.0]))
    assert rp2.tolist() == [0, 2, 4] and c2.tolist() == [0, 1, 0, 1] and v2.tolist() == [-3.0, 1.0, 1.0, -4.0]


def test_bad_entry_index_and_row_pointers_are_rejected():
    """An index past the entry list, a first row pointer other than 0 and decreasing
    row pointers return HM_EINVAL from every entry point that reads them."""
    ii = np.array([0, 1, 1], np.int32)
    jj = np.array([1, 0, 0], np.int32)
    vv = np.ones(3)
    with pytest.raises(hmat.HMError) as e:  # index 3 of a 3-entry list
        hmat.ilu_assemble(2, np.array([0, 3]), ii, jj, vv, np.zeros(2))
    assert e.value.status == hmat.HM_EINVAL
    L = hmat.lib()
    idx = np.array([0, 2], np.int64)
    rp = np.empty(3, np.int64)
    col = np.empty(4, np.int32)
    val = np.empty(4)
    nnz = ctypes.c_int64()
    st = L.hm_ilu_assemble(2, 2, 2, idx.ctypes.data, ii.ctypes.data, jj.ctypes.data, vv.ctypes.data,
                           np.zeros(2).ctypes.data, None, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                           ctypes.byref(nnz))
    assert st == hmat.HM_EINVAL  # index 2 with n_entries = 2
    bad_first = np.array([1, 2, 3], np.int64)  # rowptr[0] != 0
    c3 = np.array([0, 0, 1], np.int32)
    leaf = np.array([0, 1], np.int32)
    for call in (lambda: hmat.ilu0_factor(bad_first, c3, np.ones(3)),
                 lambda: hmat.ilu_levels(bad_first, c3),
                 lambda: hmat.ilu_leaf_colours(bad_first, c3, leaf, 2),
                 lambda: hmat.ilu_leaf_colours(np.array([0, 2, 1], np.int64), c3, leaf, 2)):
        with pytest.raises(hmat.HMError) as e:
            call()
        assert e.value.status == hmat.HM_EINVAL
