"""Oracle of the sparse approximation of the mechanical block and of its incomplete-LU
preconditioner (Sec. 3.3.1).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path; it shares no
code with the CUDA library.

Sec. 3.3.1 replaces A11 = E + C^ep, for preconditioning, by a sparse matrix: the
consistent tangent C^ep (block diagonal) plus the fraction p (0 < p <= 1, 0.01 by
default) of the entries of the full-rank (near-field) blocks of the hierarchical E that
have the largest absolute value; the inverse of that sparse matrix is applied through an
incomplete LU factorization.  Readings taken where the paper is silent:
  * C^ep is diag(k) or a block-diagonal matrix of 3x3 element blocks (the tangent
    A = E - diag(k) - C^ep - shift I); all of C^ep's entries belong to the pattern;
  * the near-field entries are those of the inadmissible leaf pairs of the block
    partition (eta), whatever the compression later does with the admissible blocks;
  * the selection is global over all near-field entries: the ceil(p n) largest in
    absolute value, ties broken by (row, column) in cluster DOF order, so it is unique;
  * the diagonal always belongs to the pattern (it carries -k even where E's own
    diagonal entry was not selected), so the factorization has its pivots in place;
  * the incomplete factorization is ILU(0) on that pattern -- no fill, no pivoting --
    with the DOFs in cluster order (the order of the near-field blocks), or, for a
    shallower dependency graph of the triangular solves, in a leaf-colour order: the
    leaves coloured greedily in leaf order (the smallest colour none of its already
    coloured neighbours holds; two leaves are neighbours when the pattern couples them)
    and listed colour by colour, leaf order within a colour, cluster order within a
    leaf.
Plain FP64 Python over dictionaries of rows: for the small cases of the tests.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def cluster_dofs(tree):
    """DOF indices in cluster order (position -> user DOF)."""
    return O.dof_index(tree.perm)


def near_entries(Emat, tree, eta=2.0):
    """Every entry of the near (inadmissible leaf-pair) blocks of the dense E, numbered in
    cluster DOF order: arrays (i, j, v)."""
    cd = cluster_dofs(tree)
    pos = np.empty(cd.size, dtype=np.int64)
    pos[cd] = np.arange(cd.size)
    near, _ = O.block_partition(tree, eta)
    I, J, V = [], [], []
    for s, t in near:
        rs = O.dof_index(tree.perm[tree.begin[s]:tree.end[s]])
        rt = O.dof_index(tree.perm[tree.begin[t]:tree.end[t]])
        blk = Emat[np.ix_(rs, rt)]
        ii, jj = np.meshgrid(pos[rs], pos[rt], indexing="ij")
        I.append(ii.ravel())
        J.append(jj.ravel())
        V.append(blk.ravel())
    return np.concatenate(I), np.concatenate(J), np.concatenate(V)


def select_largest(i, j, v, p):
    """The ceil(p n) entries of largest |v|, ties by (i, j) ascending; returned in that
    order."""
    if not (0.0 < p <= 1.0):
        raise ValueError("p must lie in (0, 1]")
    m = int(math.ceil(p * v.size))
    order = np.lexsort((j, i, -np.abs(v)))[:m]
    return i[order], j[order], v[order]


def sparse_tangent(Emat, tree, k=None, p=0.01, eta=2.0, shift=0.0, cep=None):
    """The sparse approximation of A = E - diag(k) - C^ep - shift I in cluster DOF order,
    as a list of rows {column: value}; k per element (on its 3 DOFs) or per DOF; cep the
    block-diagonal consistent tangent, (N, 3, 3) in user element order, which enters with
    every entry of its blocks (Sec. 3.3.1: the sparse matrix is C^ep plus the selected
    near-field entries)."""
    n = Emat.shape[0]
    i, j, v = select_largest(*near_entries(Emat, tree, eta), p)
    rows = [dict() for _ in range(n)]
    for a, b, x in zip(i.tolist(), j.tolist(), v.tolist()):
        rows[a][b] = x
    d = np.full(n, float(shift))
    if k is not None:
        k = np.asarray(k, dtype=np.float64)
        kd = np.repeat(k, 3) if k.size * 3 == n else k
        d += kd[cluster_dofs(tree)]
    for a in range(n):
        rows[a][a] = rows[a].get(a, 0.0) - d[a]
    if cep is not None:
        cep = np.asarray(cep, dtype=np.float64).reshape(n // 3, 3, 3)
        perm = np.asarray(tree.perm)
        for q in range(n // 3):            # cluster position q holds user element perm[q]
            for r in range(3):
                for c in range(3):
                    a, b = 3 * q + r, 3 * q + c
                    rows[a][b] = rows[a].get(b, 0.0) - cep[perm[q], r, c]
    return rows


def to_dense(rows):
    n = len(rows)
    M = np.zeros((n, n))
    for a, r in enumerate(rows):
        for b, x in r.items():
            M[a, b] = x
    return M


def ilu0(rows):
    """ILU(0): L unit lower and U upper triangular, both confined to the pattern of the
    matrix, with (L U)_ab = A_ab at every (a, b) of the pattern.  Row by row: each entry
    left of the diagonal becomes a multiplier l_ab = a_ab / u_bb, and row b of U times
    that multiplier is taken off the entries of row a that lie in the pattern; products
    falling outside the pattern are dropped.  Returns (L, U) as rows (L without its unit
    diagonal)."""
    n = len(rows)
    W = [dict(r) for r in rows]
    for a in range(n):
        if a not in W[a]:
            raise ValueError("ILU(0): the diagonal is not in the pattern")
    for a in range(n):
        ra = W[a]
        for b in sorted(c for c in ra if c < a):
            ub = W[b][b]
            if ub == 0.0:
                raise ZeroDivisionError("ILU(0): zero pivot")
            lab = ra[b] / ub
            ra[b] = lab
            for c, x in W[b].items():
                if c > b and c in ra:
                    ra[c] -= lab * x
    L = [{c: x for c, x in W[a].items() if c < a} for a in range(n)]
    U = [{c: x for c, x in W[a].items() if c >= a} for a in range(n)]
    return L, U


def ilu0_solve(L, U, r):
    """z = (L U)^-1 r: forward substitution with the unit lower factor, then backward
    substitution with the upper one."""
    n = len(L)
    y = np.array(r, dtype=np.float64)
    for a in range(n):
        y[a] -= sum(x * y[c] for c, x in L[a].items())
    z = y.copy()
    for a in range(n - 1, -1, -1):
        z[a] = (z[a] - sum(x * z[c] for c, x in U[a].items() if c > a)) / U[a][a]
    return z


def leaf_of_position(tree):
    """Leaf ordinal (in tree.leaves() order) of every cluster-order DOF position."""
    lv = tree.leaves()
    out = np.empty(3 * tree.perm.size, dtype=np.int64)
    for li, q in enumerate(lv):
        out[3 * tree.begin[q]:3 * tree.end[q]] = li
    return out


def leaf_colours(rows, tree):
    """Greedy colouring of the leaves in leaf order: each takes the smallest colour that
    none of its already coloured neighbours (leaves the pattern couples it with, in
    either direction) holds."""
    leaf = leaf_of_position(tree)
    nl = int(leaf.max()) + 1
    nbr = [set() for _ in range(nl)]
    for a, r in enumerate(rows):
        for c in r:
            if leaf[c] != leaf[a]:
                nbr[leaf[a]].add(int(leaf[c]))
                nbr[leaf[c]].add(int(leaf[a]))
    colour = [-1] * nl
    for l in range(nl):
        used = {colour[m] for m in nbr[l] if colour[m] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[l] = c
    return np.array(colour, dtype=np.int64)


def colour_order(rows, tree):
    """Cluster-order positions listed colour by colour (leaf order within a colour,
    cluster order within a leaf): new position -> cluster position."""
    leaf = leaf_of_position(tree)
    col = leaf_colours(rows, tree)
    return np.lexsort((np.arange(leaf.size), leaf, col[leaf]))


def permute_rows(rows, order):
    """The rows renumbered so that new position q holds old position order[q]."""
    newpos = np.empty(len(rows), dtype=np.int64)
    newpos[order] = np.arange(len(rows))
    return [{int(newpos[c]): x for c, x in rows[int(o)].items()} for o in order]


def solve_depth(rows):
    """Levels of the lower triangular solve: row a waits for every earlier row its
    pattern names."""
    lev = np.zeros(len(rows), dtype=np.int64)
    for a, r in enumerate(rows):
        deps = [c for c in r if c < a]
        lev[a] = 1 + (lev[deps].max() if deps else 0)
    return int(lev.max()) if len(rows) else 0


def ilu_preconditioner(Emat, tree, k=None, p=0.01, eta=2.0, shift=0.0, ordering="cluster", cep=None):
    """M^-1 for vectors in user DOF order: permute to the factorization order (cluster
    order, or the leaf-colour order), apply (L U)^-1 of the sparse approximation, permute
    back.  Returns (apply, nnz of the pattern)."""
    rows = sparse_tangent(Emat, tree, k, p, eta, shift, cep)
    cd = cluster_dofs(tree)
    if ordering == "cluster":
        order = np.arange(len(rows))
    elif ordering == "colour":
        order = colour_order(rows, tree)
    else:
        raise ValueError("ordering must be 'cluster' or 'colour'")
    L, U = ilu0(permute_rows(rows, order))
    user = cd[order]  # factorization position -> user DOF
    nnz = sum(len(r) for r in rows)

    def apply(r):
        z = np.empty_like(r)
        z[user] = ilu0_solve(L, U, r[user])
        return z

    return apply, nnz
