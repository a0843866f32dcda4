"""Pins of the oracle's learned block-Jacobi correction (oracle/learned.py) against what
the mathematics fixes: central finite differences of the loss (h = 1e-6, FP64), the
identity network (zero output layer) and its closed-form gradient, the quadratic
minimiser of the per-(leaf, component) loss, Adam's first step in closed form, feature
invariants and special cases, and the training statistics against least squares."""
import math

import numpy as np
import pytest

from oracle import learned as Lr
from oracle import oracle as O
from paper_2605_14397_gb300 import synth

H = 6


def random_problem(seed, S=7):
    rng = np.random.default_rng(seed)
    theta = rng.normal(size=Lr.param_count(H)) * 0.7
    X = rng.normal(size=(S, Lr.N_FEATURES))
    qxy = rng.normal(size=(S, 3))
    qyy = rng.uniform(0.2, 2.0, size=(S, 3))
    qxx = rng.uniform(0.5, 3.0, size=(S, 3))
    return theta, X, np.hstack([qxy, qyy, qxx])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    theta, X, Q = random_problem(seed)
    _, g = Lr.loss_and_grad(theta, H, X, Q)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (Lr.loss_and_grad(tp, H, X, Q)[0] - Lr.loss_and_grad(tm, H, X, Q)[0]) / (2 * h)
    assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)


def test_zero_output_layer_is_block_jacobi():
    theta, X, Q = random_problem(3)
    W1, b1, W2, b2, W3, b3 = Lr.unpack(theta, H)
    t0 = Lr.pack(W1, b1, W2, b2, np.zeros_like(W3), np.zeros_like(b3))
    d, _ = Lr.forward(t0, H, X)
    assert np.all(d == 1.0)
    loss, g = Lr.loss_and_grad(t0, H, X, Q)
    qxy, qyy, qxx = Q[:, 0:3], Q[:, 3:6], Q[:, 6:9]
    assert loss == pytest.approx((qxx - 2 * qxy + qyy).sum(), rel=1e-14)
    gW1, gb1, gW2, gb2, gW3, gb3 = Lr.unpack(g, H)
    for z in (gW1, gb1, gW2, gb2):
        assert np.all(z == 0.0)
    # dloss/db3_a = sum_s 2 (q_yy - q_xy) * 0.5 (d/do at o = 0 is 1/2)
    assert np.allclose(gb3, (qyy - qxy).sum(axis=0), rtol=1e-13)


def test_quadratic_minimiser_per_component():
    # one sample; the output bias alone sets d = q_xy / q_yy, where the loss is minimal
    qxy = np.array([0.9, 1.1, 0.7])
    qyy = np.array([1.0, 1.0, 1.0])
    qxx = np.array([2.0, 3.0, 1.0])
    Q = np.hstack([qxy, qyy, qxx])[None, :]
    dstar = qxy / qyy
    theta = np.zeros(Lr.param_count(H))
    W1, b1, W2, b2, W3, b3 = Lr.unpack(theta, H)
    b3 = np.arctanh(2.0 * (dstar - 1.0))
    t = Lr.pack(W1, b1, W2, b2, W3, b3)
    loss, g = Lr.loss_and_grad(t, H, np.zeros((1, Lr.N_FEATURES)), Q)
    assert loss == pytest.approx((qxx - qxy ** 2 / qyy).sum(), rel=1e-13)
    assert np.abs(Lr.unpack(g, H)[5]).max() < 1e-13


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    theta = rng.normal(size=20)
    g = rng.normal(size=20)
    lr = 1e-3
    t1, m, v = Lr.adam_step(theta, g, np.zeros(20), np.zeros(20), 1, lr)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def _tree_arrays(el, leaf):
    T = O.cluster_tree(el, leaf)
    lv = T.leaves()
    return T.perm, np.array([T.begin[q] for q in lv]), np.array([T.end[q] for q in lv])


def test_features_special_cases():
    el = synth.config_penny(16)
    perm, begin, end = _tree_arrays(el, 16)
    h = 2.0 / 16
    k = np.full(el.N, 0.3 / h)  # k h / E = 0.3 everywhere
    F = Lr.leaf_features(el, k, 1.0, perm, begin, end)
    kap = math.log10(0.3 + 1e-6)
    assert np.allclose(F[:, 0], kap) and np.allclose(F[:, 2], kap) and np.allclose(F[:, 3], kap)
    assert np.allclose(F[:, 1], 0.0, atol=1e-15)
    assert np.all(F[:, 4] == 1.0)  # 0.3 < 0.5: soft
    assert np.allclose(F[:, 5], np.log10(end - begin))
    assert np.allclose(F[:, 6], 1.0)  # planar
    assert np.allclose(F[:, 7], math.log10(1001.0))  # no other plane
    # a rigid translation changes nothing
    moved = synth.config_penny(16)
    moved.c = moved.c + np.array([3.0, -2.0, 5.0])
    assert np.allclose(Lr.leaf_features(moved, k, 1.0, perm, begin, end), F, atol=1e-12)


def test_features_two_planes_distance_and_mixture():
    el = synth.config_crack_fault(h=0.25)
    perm, begin, end = _tree_arrays(el, 8)
    rng = np.random.default_rng(5)
    k = np.exp(rng.uniform(math.log(1e-3), math.log(1e2), size=el.N)) / 0.25
    F = Lr.leaf_features(el, k, 1.0, perm, begin, end)
    assert np.all(F[:, 7] < math.log10(1001.0))  # every leaf sees the other plane
    s = k * 0.25
    for l in range(len(begin)):
        idx = perm[begin[l]:end[l]]
        assert F[l, 4] == pytest.approx(np.mean(s[idx] < 0.5))
        assert F[l, 2] <= F[l, 0] <= F[l, 3]


def test_stats_give_least_squares_scaling():
    el = synth.config_penny(12)
    perm, begin, end = _tree_arrays(el, 16)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 3 * el.N))
    y = rng.normal(size=(2, 3 * el.N))
    S = Lr.leaf_stats(x, y, perm, begin, end)
    for l in range(len(begin)):
        idx = perm[begin[l]:end[l]]
        for a in range(3):
            dofs = 3 * idx + a
            ls = np.linalg.lstsq(y[:, dofs].reshape(-1, 1), x[:, dofs].reshape(-1), rcond=None)[0][0]
            assert S[l, a] / S[l, 3 + a] == pytest.approx(ls, rel=1e-12)
    Q = Lr.samples([S, 2 * S])
    assert Q[:, 6:9].sum() == pytest.approx(1.0)


def test_two_level_corrections_cannot_beat_block_jacobi_on_the_tangent():
    """What a learned correction of leaf block-Jacobi B could gain on the tangent of a
    crack crossing a fault (k log-uniform in [1e-3, 1e2] E/h): B^-1 A has all its
    eigenvalues in a ring around 1 (|lambda| in [0.05, 2]), and a two-level correction
    with the ideal coarse space of three columns per leaf -- the leaf restrictions of the
    slowest modes of B^-1 A, an upper bound for any learned one -- saves at most two
    GMRES iterations while the multiplicative form costs a second product per iteration;
    the additive form saves none."""
    import scipy.linalg as sla
    from oracle import oracle as O
    from paper_2605_14397_gb300 import synth
    h = 0.15
    el = synth.config_crack_fault(h=h)
    T = O.cluster_tree(el, 64)
    dofs = [O.dof_index(T.perm[T.begin[q]:T.end[q]]) for q in T.leaves()]
    A = O.tangent_dense(O.dense_matrix(el, 1.0, 0.25), synth.k_loguniform(el.N, 1605001, E=1.0, h=h))
    inv = O.block_jacobi_inverses(A, T)
    b = synth.rhs_normal(A.shape[0], 1605008)
    _, it_bj, ok, _ = O.gmres(lambda v: A @ v, b, lambda r: O.apply_block_jacobi(inv, r), tol=1e-8)
    BA = np.zeros_like(A)
    for d, Bi in inv:
        BA[d] = Bi @ A[d]
    w, V = np.linalg.eig(BA)
    assert np.abs(w).min() > 0.04 and np.abs(w).max() < 2.0
    slow = np.real(V[:, np.argsort(np.abs(w))[:12 * len(dofs)]])
    Z = np.zeros((A.shape[0], 3 * len(dofs)))
    for li, d in enumerate(dofs):
        Z[d, 3 * li:3 * li + 3] = np.linalg.svd(slow[d], full_matrices=False)[0][:, :3]
    lu = sla.lu_factor(Z.T @ A @ Z)
    coarse = lambda r: Z @ sla.lu_solve(lu, Z.T @ r)
    bj = lambda r: O.apply_block_jacobi(inv, r)

    def mult(r):
        y = bj(r)
        return y + coarse(r - A @ y)

    _, it_add, ok_a, _ = O.gmres(lambda v: A @ v, b, lambda r: bj(r) + coarse(r), tol=1e-8)
    _, it_mul, ok_m, _ = O.gmres(lambda v: A @ v, b, mult, tol=1e-8)
    assert ok and ok_a and ok_m
    assert it_add >= it_bj and it_bj - 2 <= it_mul <= it_bj
    assert 2 * it_mul > it_bj  # products: two per multiplicative iteration


def test_near_offdiag_partitions_E():
    """N holds exactly the near-field entries off the diagonal leaf blocks: with the
    diagonal leaf blocks and the admissible blocks it rebuilds E entry by entry, each entry
    once (the block partition covers the index square once)."""
    el = synth.config_crack_fault(h=0.25)
    T = O.cluster_tree(el, 16)
    Em = O.dense_matrix(el, 1.0, 0.25)
    Nm = Lr.near_offdiag(Em, T)
    near, far = O.block_partition(T, 2.0)
    cover = np.zeros(Em.shape)
    rebuilt = Nm.copy()
    for q in T.leaves():
        d = O.dof_index(T.perm[T.begin[q]:T.end[q]])
        rebuilt[np.ix_(d, d)] += Em[np.ix_(d, d)]
        cover[np.ix_(d, d)] += 1
    for s, t in far:
        rs = O.dof_index(T.perm[T.begin[s]:T.end[s]])
        ct = O.dof_index(T.perm[T.begin[t]:T.end[t]])
        rebuilt[np.ix_(rs, ct)] += Em[np.ix_(rs, ct)]
        cover[np.ix_(rs, ct)] += 1
    cover += (Nm != 0)
    assert np.array_equal(rebuilt, Em)
    assert cover.max() == 1 and len(near) > len(T.leaves())


def test_near_correction_is_a_first_order_neumann_term():
    """With N = 0 the near correction is B^-1; on A = B + eps N (block-diagonal B, no far
    part) y - B^-1 N y with d = gamma = 1 is the first Neumann approximation of A^-1:
    its error falls like eps^2."""
    rng = np.random.default_rng(9)
    n = 12
    perm = np.arange(4)
    begin, end = [0, 2], [2, 4]
    B = np.zeros((n, n))
    for lo, hi in ((0, 6), (6, 12)):
        B[lo:hi, lo:hi] = rng.normal(size=(6, 6)) + 6 * np.eye(6)
    N0 = rng.normal(size=(n, n))
    N0[:6, :6] = 0
    N0[6:, 6:] = 0
    Binv = np.linalg.inv(B)
    d = np.ones((2, 3))
    r = rng.normal(size=n)
    z0 = Lr.apply_near(d, 1.0, r, np.zeros((n, n)), perm, begin, end, lambda v: Binv @ v)
    assert np.allclose(z0, Binv @ r, rtol=1e-14, atol=0)
    errs = []
    for eps in (1e-2, 1e-3):
        A = B + eps * N0
        z = Lr.apply_near(d, 1.0, r, eps * N0, perm, begin, end, lambda v: Binv @ v)
        errs.append(np.linalg.norm(z - np.linalg.solve(A, r)))
    assert errs[1] < 2e-2 * errs[0]  # quadratic: a 10x smaller eps gives ~100x less error


def test_near_stats_give_the_least_squares_damping():
    """The (leaf, component) minimiser q_xy / q_yy of the near statistics is the least
    squares fit of d w to y - x on that group."""
    el = synth.config_penny(10)
    T = O.cluster_tree(el, 16)
    Em = O.dense_matrix(el, 1.0, 0.25)
    k = synth.k_loguniform(el.N, 3, h=0.2)
    A = O.tangent_dense(Em, k)
    inv = O.block_jacobi_inverses(A, T)
    bj = lambda v: O.apply_block_jacobi(inv, v)
    Nm = Lr.near_offdiag(Em, T)
    b = synth.rhs_normal(A.shape[0], 4)
    x = np.linalg.solve(A, b)
    leaves = T.leaves()
    begin = [T.begin[q] for q in leaves]
    end = [T.end[q] for q in leaves]
    S = Lr.near_stats(x, b, Nm, T.perm, begin, end, bj)
    y = bj(b)
    w = bj(Nm @ y)
    for l in range(len(leaves)):
        idx = T.perm[begin[l]:end[l]]
        for a in range(3):
            dofs = 3 * idx + a
            ls = np.linalg.lstsq(w[dofs, None], (y - x)[dofs], rcond=None)[0][0]
            assert S[l, a] / S[l, 3 + a] == pytest.approx(ls, rel=1e-12)


@pytest.mark.parametrize("seed", [1606000, 1606001])
def test_per_leaf_scaling_of_the_near_correction_has_no_headroom(seed):
    """What the network of the near correction M = B^-1 - gamma D B^-1 N B^-1 can add
    beyond a constant damping, on the tangent of a crack crossing a fault (h = 0.15,
    16 leaves, k log-uniform): the damped correction with D = I cuts GMRES iterations by
    a third against block-Jacobi for the best gamma in 0.6..1.0, and the per-(leaf,
    component) scaling that minimises sum ||r - A M r||^2 over 8 probe vectors r -- the
    optimum of a loss that sees the spectrum of A M, fitted on the very system it is
    tested on -- saves at most one iteration more."""
    h = 0.15
    el = synth.config_crack_fault(h=h)
    Em = O.dense_matrix(el, 1.0, 0.25)
    T = O.cluster_tree(el, 64)
    perm, begin, end = _tree_arrays(el, 64)
    Nm = Lr.near_offdiag(Em, T)
    nl, n = len(begin), 3 * el.N
    A = O.tangent_dense(Em, synth.k_loguniform(el.N, seed, E=1.0, h=h))
    inv = O.block_jacobi_inverses(A, T)
    bj = lambda v: O.apply_block_jacobi(inv, v)
    b = synth.rhs_normal(n, seed)

    def iters(M):
        _, it, ok, _ = O.gmres(lambda v: A @ v, b, M, tol=1e-8, restart=50)
        assert ok
        return it
    it_bj = iters(bj)
    it_d1 = min(iters(lambda r, g=g: Lr.apply_near(np.ones((nl, 3)), g, r, Nm, perm, begin, end, bj))
                for g in (0.6, 0.7, 0.8, 0.9, 1.0))
    assert it_d1 <= 0.7 * it_bj
    # A M r = A y - sum_(l, a) d_(l, a) A (u restricted to leaf l, component a)
    rng = np.random.default_rng(5)
    rows, rhs = [], []
    for _ in range(8):
        r = rng.normal(size=n)
        y = bj(r)
        u = bj(Nm @ y)
        cols = []
        for l in range(nl):
            for a in range(3):
                q = 3 * perm[begin[l]:end[l]] + a
                v = np.zeros(n)
                v[q] = u[q]
                cols.append(A @ v)
        rows.append(np.stack(cols, 1))
        rhs.append(A @ y - r)
    d = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0].reshape(nl, 3)
    it_opt = iters(lambda r: Lr.apply_near(d, 1.0, r, Nm, perm, begin, end, bj))
    assert it_opt >= it_d1 - 1
