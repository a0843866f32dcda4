"""Plain, slow, FP64 CPU oracle of the H-matrix DD-BEM hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline leg; never by the product path.  It shares no code with the CUDA library.

Contents, each following the passage it cites:
  * influence coefficients of constant-DD rectangles and triangles (Sec. 3.1, eq.
    TractionBIE-general and eq. ElasSystem; the C part in ddm_oracle.c),
  * the dense operator E and dense products E x (eq. ElasSystem),
  * the centroid cluster tree and the block partition that the H-matrix uses
    (Sec. 3.1: near field kept dense, far field low rank; the split and admissibility
    rules are the readings stated in the design notes: longest-axis median bisection,
    min(diam) <= eta dist on vertex boxes),
  * the tangent operator A = E - diag(k) (eq. jac_mech with C^ep = diag(k)),
  * leaf block-Jacobi (the point-Jacobi of Sec. 3.3.1 taken per leaf) and the 3x3
    point Jacobi itself,
  * restarted right-preconditioned GMRES(m) with classical Gram-Schmidt applied twice
    (the Krylov solve of the A11 system, Sec. 3.3.1),
  * Sneddon's and Segedin's penny-crack openings (the closed forms used as pins).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.c_int64
        d = ctypes.c_double
        g = [dp, dp, dp, dp, dp, dp, i32p, dp]
        L.orc_blocks.restype = i64
        L.orc_blocks.argtypes = [i64] + g + [d, d, i64, ip, ip, dp]
        L.orc_dense_rows.restype = i64
        L.orc_dense_rows.argtypes = [i64] + g + [d, d, i64, ip, dp]
        L.orc_dense_matvec_rows.restype = i64
        L.orc_dense_matvec_rows.argtypes = [i64] + g + [d, d, i64, ip, i64, dp, dp]
        L.orc_tri_phi_derivatives.restype = ctypes.c_int
        L.orc_tri_phi_derivatives.argtypes = [dp, dp, dp, dp]
        L.orc_influence_tri.restype = ctypes.c_int
        L.orc_influence_tri.argtypes = [dp] * 9 + [d, d, dp]
        L.orc_phi_derivatives.restype = ctypes.c_int
        L.orc_phi_derivatives.argtypes = [dp, d, d, dp, dp]
        L.orc_influence.restype = ctypes.c_int
        L.orc_influence.argtypes = [dp] * 8 + [d, d, d, d, dp]
        _LIB = L
    return _LIB


def _p(a, dtype=np.float64):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double if dtype == np.float64 else ctypes.c_int64))


def _geom(el):
    """ctypes pointers of the geometry: c, s1, s2, n, a, b, then shape and the triangle
    vertices (NULL when every element is a rectangle); the arrays are kept alive on the
    returned list."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (el.c, el.s1, el.s2, el.n, el.a, el.b)]
    ptrs = [_p(x) for x in arrs]
    shape = getattr(el, "shape", None)
    if shape is not None and np.any(np.asarray(shape) != 0):
        sh = np.ascontiguousarray(shape, dtype=np.int32)
        tri = np.ascontiguousarray(el.tri, dtype=np.float64)
        arrs += [sh, tri]
        ptrs += [sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _p(tri)]
    else:
        ptrs += [None, None]
    return _Geom(arrs, ptrs)


class _Geom(list):
    def __init__(self, arrs, ptrs):
        super().__init__(ptrs)
        self.arrs = arrs


def set_threads(n: int | None):
    """Number of OpenMP threads the oracle uses (None: all cores)."""
    if n is None:
        os.environ.pop("OMP_NUM_THREADS", None)
    else:
        os.environ["OMP_NUM_THREADS"] = str(int(n))


# ------------------------------------------------------------------ influence coefficients

def shear_modulus(E, nu):
    return E / (2.0 * (1.0 + nu))


def influence_blocks(el, E, nu, ri, sj):
    """3x3 blocks E_{ri[p], sj[p]} (receiver frame rows, source frame columns)."""
    g = _geom(el)
    ri = np.ascontiguousarray(ri, dtype=np.int64)
    sj = np.ascontiguousarray(sj, dtype=np.int64)
    out = np.empty((ri.size, 9))
    lib().orc_blocks(el.N, *g, float(E), float(nu), ri.size,
                     _p(ri, np.int64), _p(sj, np.int64), _p(out))
    return out.reshape(-1, 3, 3)


def influence_point(xr, rframe, cs, sframe, a, b, E, nu):
    """Block for an arbitrary receiver point and frame (frames as (s1, s2, n))."""
    vecs = [np.ascontiguousarray(v, dtype=np.float64) for v in
            (xr, rframe[0], rframe[1], rframe[2], cs, sframe[0], sframe[1], sframe[2])]
    out = np.empty(9)
    st = lib().orc_influence(*[_p(v) for v in vecs], float(a), float(b),
                             shear_modulus(E, nu), float(nu), _p(out))
    return st, out.reshape(3, 3)


def phi_derivatives(x, a, b):
    x = np.ascontiguousarray(x, dtype=np.float64)
    d2 = np.empty(9)
    d3 = np.empty(27)
    st = lib().orc_phi_derivatives(_p(x), float(a), float(b), _p(d2), _p(d3))
    return st, d2.reshape(3, 3), d3.reshape(3, 3, 3)


def tri_phi_derivatives(x, tv):
    """phi's second and third derivatives for the triangle with vertices tv (3 x 2, in
    its plane frame) at the point x of that frame (edge integrals by quadrature)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    tv = np.ascontiguousarray(tv, dtype=np.float64).reshape(6)
    d2 = np.empty(9)
    d3 = np.empty(27)
    st = lib().orc_tri_phi_derivatives(_p(x), _p(tv), _p(d2), _p(d3))
    return st, d2.reshape(3, 3), d3.reshape(3, 3, 3)


def influence_point_tri(xr, rframe, cs, sframe, V, E, nu):
    """Block for an arbitrary receiver point and frame from the triangle with vertices V
    (3 x 3, global) collocated at cs with frame sframe."""
    vecs = [np.ascontiguousarray(v, dtype=np.float64) for v in
            (xr, rframe[0], rframe[1], rframe[2], cs, sframe[0], sframe[1], sframe[2])]
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(9)
    out = np.empty(9)
    st = lib().orc_influence_tri(*[_p(v) for v in vecs], _p(V), shear_modulus(E, nu), float(nu), _p(out))
    return st, out.reshape(3, 3)


def dense_matrix(el, E, nu):
    """The dense collocation matrix E (3N x 3N), DOF order (s1, s2, n) per element."""
    return dense_rows(el, E, nu, np.arange(el.N))


def dense_rows(el, E, nu, rows):
    g = _geom(el)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((3 * rows.size, 3 * el.N))
    bad = lib().orc_dense_rows(el.N, *g, float(E), float(nu), rows.size,
                               _p(rows, np.int64), _p(out))
    if bad:
        raise ValueError("%d receiver/source pairs are singular (receiver on a source edge)" % bad)
    return out


def dense_matvec_rows(el, E, nu, x, rows=None):
    """y = E[rows, :] x without storing E; x of shape (3N,) or (nrhs, 3N)."""
    g = _geom(el)
    if rows is None:
        rows = np.arange(el.N)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    X = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    nrhs = X.shape[0]
    Y = np.empty((nrhs, 3 * rows.size))
    bad = lib().orc_dense_matvec_rows(el.N, *g, float(E), float(nu), rows.size,
                                      _p(rows, np.int64), nrhs, _p(X), _p(Y))
    if bad:
        raise ValueError("%d receiver/source pairs are singular" % bad)
    return Y[0] if np.ndim(x) == 1 else Y


# ------------------------------------------------------------------ cluster tree (Sec. 3.1)

class ClusterTree:
    """Binary cluster tree over element centroids.

    Nodes are numbered in depth-first pre-order (root 0, then the left subtree, then the
    right one).  perm[k] is the user index of the element at cluster position k; node q
    owns positions begin[q] <= k < end[q]."""

    def __init__(self, perm, begin, end, left, right, lo, hi):
        self.perm = perm
        self.begin = begin
        self.end = end
        self.left = left
        self.right = right
        self.lo = lo
        self.hi = hi

    @property
    def n_nodes(self):
        return len(self.begin)

    def is_leaf(self, q):
        return self.left[q] < 0

    def leaves(self):
        return [q for q in range(self.n_nodes) if self.left[q] < 0]


def element_vertex_boxes(el):
    """Per-element bounding box of its vertices: the 4 rectangle vertices
    c +- a s1 +- b s2, or the 3 given vertices of a triangle."""
    lo = np.full((el.N, 3), np.inf)
    hi = np.full((el.N, 3), -np.inf)
    for sa in (-1.0, 1.0):
        for sb in (-1.0, 1.0):
            v = el.c + (sa * el.a)[:, None] * el.s1 + (sb * el.b)[:, None] * el.s2
            lo = np.minimum(lo, v)
            hi = np.maximum(hi, v)
    shape = getattr(el, "shape", None)
    if shape is not None and np.any(np.asarray(shape) == 1):
        t = np.asarray(shape) == 1
        V = np.asarray(el.tri)[t].reshape(-1, 3, 3)
        lo[t] = V.min(axis=1)
        hi[t] = V.max(axis=1)
    return lo, hi


def cluster_tree(el, leaf_size=64):
    """Recursive bisection: split a cluster with more than leaf_size elements along the
    longest axis of its centroid bounding box at the median (the first n//2 elements in
    the order (coordinate, user index) go left)."""
    c = el.c
    vlo, vhi = element_vertex_boxes(el)
    perm = np.arange(el.N, dtype=np.int64)
    begin, end, left, right, lo, hi = [], [], [], [], [], []

    def make(b, e):
        q = len(begin)
        begin.append(b)
        end.append(e)
        left.append(-1)
        right.append(-1)
        idx = perm[b:e]
        lo.append(vlo[idx].min(axis=0))
        hi.append(vhi[idx].max(axis=0))
        n = e - b
        if n > leaf_size and n > 1:
            cc = c[idx]
            ext = cc.max(axis=0) - cc.min(axis=0)
            axis = int(np.argmax(ext))
            order = np.lexsort((idx, cc[:, axis]))  # primary: coordinate, then index
            perm[b:e] = idx[order]
            m = b + n // 2
            left[q] = make(b, m)
            right[q] = make(m, e)
        return q

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        make(0, el.N)
    finally:
        sys.setrecursionlimit(old)
    return ClusterTree(perm, np.array(begin, dtype=np.int64), np.array(end, dtype=np.int64),
                       np.array(left, dtype=np.int64), np.array(right, dtype=np.int64),
                       np.array(lo), np.array(hi))


def _diam(lo, hi):
    d0, d1, d2 = float(hi[0] - lo[0]), float(hi[1] - lo[1]), float(hi[2] - lo[2])
    return math.sqrt(d0 * d0 + d1 * d1 + d2 * d2)


def _dist(lo1, hi1, lo2, hi2):
    d = []
    for k in range(3):
        g = max(0.0, float(lo2[k] - hi1[k]), float(lo1[k] - hi2[k]))
        d.append(g)
    return math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])


def admissible(tree, s, t, eta):
    ds = _diam(tree.lo[s], tree.hi[s])
    dt = _diam(tree.lo[t], tree.hi[t])
    dist = _dist(tree.lo[s], tree.hi[s], tree.lo[t], tree.hi[t])
    return dist > 0.0 and min(ds, dt) <= eta * dist


def block_partition(tree, eta=2.0):
    """Block cluster tree from (root, root): an admissible pair is a far (low-rank) block;
    a pair of leaves that is not admissible is a near (dense) block; otherwise split the
    non-leaf members (both when both are non-leaves) and recurse, children in the order
    (s0,t0), (s0,t1), (s1,t0), (s1,t1).  Returns (near, far) as lists of (s, t)."""
    near, far = [], []
    stack = [(0, 0)]
    while stack:
        s, t = stack.pop()
        if admissible(tree, s, t, eta):
            far.append((s, t))
            continue
        ls, lt = tree.is_leaf(s), tree.is_leaf(t)
        if ls and lt:
            near.append((s, t))
            continue
        cs = [s] if ls else [tree.left[s], tree.right[s]]
        ct = [t] if lt else [tree.left[t], tree.right[t]]
        kids = [(a, b) for a in cs for b in ct]
        stack.extend(reversed(kids))  # so that they pop in the stated order
    return near, far


def dof_index(perm_elems):
    """DOF indices (3e, 3e+1, 3e+2) of a list of elements."""
    e = np.asarray(perm_elems, dtype=np.int64)
    return (3 * e[:, None] + np.arange(3)[None, :]).ravel()


# ------------------------------------------------------------------ tangent + preconditioner

def tangent_dense(Emat, k=None, shift=0.0, cep=None):
    """A = E - diag(k) - C^ep - shift I (eq. jac_mech, eta/dt = shift): k per element
    (applied to its 3 DOFs) or per DOF; cep the block-diagonal consistent tangent as
    (N, 3, 3) blocks, element e's block on DOFs 3e..3e+2 (user order)."""
    A = Emat.copy()
    n = A.shape[0]
    d = np.zeros(n)
    if k is not None:
        k = np.asarray(k, dtype=np.float64)
        d += np.repeat(k, 3) if k.size * 3 == n else k
    d += shift
    A[np.arange(n), np.arange(n)] -= d
    if cep is not None:
        cep = np.asarray(cep, dtype=np.float64).reshape(n // 3, 3, 3)
        for e in range(n // 3):
            A[3 * e:3 * e + 3, 3 * e:3 * e + 3] -= cep[e]
    return A


def block_jacobi_inverses(A, tree):
    """Explicit inverse of every diagonal leaf block of A (cluster order)."""
    inv = []
    for q in tree.leaves():
        dofs = dof_index(tree.perm[tree.begin[q]:tree.end[q]])
        inv.append((dofs, np.linalg.inv(A[np.ix_(dofs, dofs)])))
    return inv


def point_jacobi_inverses(A):
    """Explicit inverse of every 3x3 diagonal block of A, one per element: the point
    Jacobi preconditioner of the A11 system (Sec. 3.3.1), an element's three DOFs
    (s1, s2, n) taken together."""
    n = A.shape[0] // 3
    return [(np.arange(3 * e, 3 * e + 3), np.linalg.inv(A[3 * e:3 * e + 3, 3 * e:3 * e + 3])) for e in range(n)]


def apply_block_jacobi(inv, r):
    z = np.zeros_like(r)
    for dofs, Binv in inv:
        z[dofs] = Binv @ r[dofs]
    return z


def gmres(apply_A, b, apply_M=None, tol=1e-8, restart=50, maxit=2000):
    """Restarted right-preconditioned GMRES(m) with x0 = 0: solve A M^-1 u = b,
    x = M^-1 u.  Arnoldi by classical Gram-Schmidt applied twice (CGS2), Givens
    rotations for the least-squares problem, stop when the Givens residual estimate
    falls to tol * ||b||; the true residual is recomputed at every restart.
    Returns (x, iterations, converged, residual history)."""
    if apply_M is None:
        apply_M = lambda v: v
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, True, [0.0]
    hist = []
    its = 0
    r = b.copy()
    beta = bnorm
    while its < maxit:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        converged = False
        for j in range(restart):
            w = apply_A(apply_M(V[j]))
            h = np.zeros(j + 1)
            for _ in range(2):  # CGS2
                c = V[:j + 1] @ w
                w = w - V[:j + 1].T @ c
                h += c
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):  # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0 or its >= maxit:
                converged = abs(g[j + 1]) <= tol * bnorm
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + apply_M(V[:j_done].T @ y)
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return x, its, True, hist
        if converged:  # estimate said converged but the true residual did not: restart
            pass
    return x, its, False, hist


def bicgstab(apply_A, b, apply_M=None, tol=1e-8, maxit=2000):
    """Right-preconditioned BiCGSTAB (van der Vorst, 1992), x0 = 0, shadow residual
    r^ = b: the Krylov method of the paper's A11 solves (Sec. 3.3.1).  Per iteration,
    p = r + beta (p - omega v), v = A M^-1 p, alpha = (r^, r) / (r^, v), s = r - alpha v,
    t = A M^-1 s, omega = (t, s) / (t, t), x += alpha M^-1 p + omega M^-1 s,
    r = s - omega t, beta = (r^, r_new) / (r^, r_old) * alpha / omega; stop when the
    recurrence's ||r|| <= tol ||b||, then check the true residual and restart from it
    if it has drifted.  Returns (x, iterations, converged)."""
    if apply_M is None:
        apply_M = lambda v: v
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, True
    its = 0
    r = b.copy()
    for _ in range(8):                       # restarts from the true residual
        rh = r.copy()
        p = np.zeros(n)
        v = np.zeros(n)
        rho = alpha = omega = 1.0
        first = True
        while its < maxit:
            rho_new = rh @ r
            if rho_new == 0.0:
                break
            beta = 0.0 if first else (rho_new / rho) * (alpha / omega)
            first = False
            rho = rho_new
            p = r + beta * (p - omega * v)
            ph = apply_M(p)
            v = apply_A(ph)
            den = rh @ v
            if den == 0.0:
                break
            alpha = rho / den
            s = r - alpha * v
            sh = apply_M(s)
            t = apply_A(sh)
            tt = t @ t
            omega = (t @ s) / tt if tt > 0.0 else 0.0
            x = x + alpha * ph + omega * sh
            r = s - omega * t
            its += 1
            if np.linalg.norm(r) <= tol * bnorm or omega == 0.0:
                break
        r = b - apply_A(x)
        if np.linalg.norm(r) <= tol * bnorm:
            return x, its, True
        if its >= maxit:
            break
    return x, its, False


# ------------------------------------------------------------------ closed-form pins

def sneddon_opening(r, E=1.0, nu=0.25, p=1.0, radius=1.0):
    """Opening of a penny crack under internal pressure p: 8(1-nu^2) p/(pi E) sqrt(R^2-r^2)."""
    return 8.0 * (1.0 - nu * nu) * p / (math.pi * E) * np.sqrt(np.maximum(radius ** 2 - r ** 2, 0.0))


def segedin_slip(r, E=1.0, nu=0.25, tau=1.0, radius=1.0):
    """Slip of a penny crack under uniform shear tau: 8(1-nu) tau/(pi mu (2-nu)) sqrt(R^2-r^2)."""
    mu = shear_modulus(E, nu)
    return 8.0 * (1.0 - nu) * tau / (math.pi * mu * (2.0 - nu)) * np.sqrt(np.maximum(radius ** 2 - r ** 2, 0.0))
