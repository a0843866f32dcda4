"""FP64 CPU oracle of the learned block-Jacobi correction.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's CPU leg).  Shares
no code with the CUDA library.

The paper preconditions its A11 system with a Jacobi preconditioner (Sec. 3.3.1) and has
nothing learned; this is the correction the library adds on top of the leaf
block-Jacobi preconditioner B of A = E - diag(k) (eq. jac_mech):

    M^-1 r = D B^-1 r,   D = diag(d_(leaf, component)),   d = 1 + 0.5 tanh(o),
    o = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3,

one scaling per leaf and DOF component (s1, s2, n) predicted by a two-hidden-layer tanh
network from eight features f of the leaf.  With W3 = 0, b3 = 0 the correction is the
identity (plain block-Jacobi).

Training fits D B^-1 to the inverse: for solved systems A x_j = b_j and y_j = B^-1 b_j,

    loss = sum over systems s of  sum_(leaf, comp) |x - d y|^2 restricted to the leaf and
           component, summed over the system's right-hand sides, / (n_systems T_s),

with T_s = sum |x|^2 of the system.  Per (leaf, component) the loss only needs the sums
S_xy, S_yy, S_xx, so a training sample is (features, q_xy[3], q_yy[3], q_xx[3]) with
q = S / (n_systems T_s), and  loss = sum_samples sum_a q_xx - 2 d_a q_xy + d_a^2 q_yy.
Parameters are updated by Adam (Kingma and Ba, 2015).
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 8
N_OUT = 3


def param_count(hidden: int) -> int:
    """W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (3 x H), b3 (3), in this order."""
    H, F = hidden, N_FEATURES
    return H * F + H + H * H + H + N_OUT * H + N_OUT


def unpack(theta, hidden):
    H, F = hidden, N_FEATURES
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == param_count(H)
    o = 0

    def take(n, shape):
        nonlocal o
        a = theta[o:o + n].reshape(shape)
        o += n
        return a

    W1 = take(H * F, (H, F))
    b1 = take(H, (H,))
    W2 = take(H * H, (H, H))
    b2 = take(H, (H,))
    W3 = take(N_OUT * H, (N_OUT, H))
    b3 = take(N_OUT, (N_OUT,))
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


# ------------------------------------------------------------------ features

def leaf_features(el, k, E, perm, begin, end):
    """Eight features per leaf (leaves given by cluster positions [begin, end) into perm):
      0-3  mean, standard deviation, min, max over the leaf of log10(k_e h_e / E + 1e-6),
           h_e = sqrt(4 a_e b_e) the element size (the stiffness relative to the
           elastic self-stiffness scale E / h),
      4    fraction of elements with k_e h_e / E < 0.5 (soft: the elastic part dominates),
      5    log10(number of elements),
      6    |mean normal| (1 for a planar leaf),
      7    log10(1 + d / hbar): d the distance from the leaf centroid to the nearest
           centroid of a leaf whose mean normal has another direction
           (|n_l . n_m| < 0.99 |n_l| |n_m|), hbar the mean element size; d = 1000 hbar
           when there is no such leaf (an intersection is near or far)."""
    k = np.asarray(k, dtype=np.float64)
    L = len(begin)
    h = np.sqrt(4.0 * el.a * el.b)
    F = np.zeros((L, N_FEATURES))
    cen = np.zeros((L, 3))
    nrm = np.zeros((L, 3))
    hbar = np.zeros(L)
    for l in range(L):
        idx = perm[begin[l]:end[l]]
        s = k[idx] * h[idx] / E
        kap = np.log10(s + 1e-6)
        mu = kap.mean()
        F[l, 0] = mu
        F[l, 1] = math.sqrt(((kap - mu) ** 2).mean())
        F[l, 2] = kap.min()
        F[l, 3] = kap.max()
        F[l, 4] = float((s < 0.5).sum()) / idx.size
        F[l, 5] = math.log10(idx.size)
        nrm[l] = el.n[idx].mean(axis=0)
        F[l, 6] = np.linalg.norm(nrm[l])
        cen[l] = el.c[idx].mean(axis=0)
        hbar[l] = h[idx].mean()
    for l in range(L):
        best = math.inf
        for m in range(L):
            if m == l:
                continue
            dot = abs(float(nrm[l] @ nrm[m]))
            if dot < 0.99 * np.linalg.norm(nrm[l]) * np.linalg.norm(nrm[m]):
                best = min(best, float(np.linalg.norm(cen[l] - cen[m])))
        d = best if math.isfinite(best) else 1000.0 * hbar[l]
        F[l, 7] = math.log10(1.0 + d / hbar[l])
    return F


# ------------------------------------------------------------------ network

def forward(theta, hidden, X):
    """Scalings d (S x 3) for feature rows X (S x 8), and the activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, hidden)
    X = np.asarray(X, dtype=np.float64)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    o = a2 @ W3.T + b3
    t = np.tanh(o)
    d = 1.0 + 0.5 * t
    return d, (X, a1, a2, t)


def loss_value(d, Q):
    """sum over samples and components of q_xx - 2 d q_xy + d^2 q_yy; Q = [q_xy | q_yy | q_xx]."""
    qxy, qyy, qxx = Q[:, 0:3], Q[:, 3:6], Q[:, 6:9]
    return float((qxx - 2.0 * d * qxy + d * d * qyy).sum())


def loss_and_grad(theta, hidden, X, Q):
    """Loss and its gradient with respect to theta (back-propagation through the
    network, chain rule layer by layer)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, hidden)
    Q = np.asarray(Q, dtype=np.float64)
    d, (X, a1, a2, t) = forward(theta, hidden, X)
    loss = loss_value(d, Q)
    qxy, qyy = Q[:, 0:3], Q[:, 3:6]
    g_d = 2.0 * (d * qyy - qxy)          # dloss/dd
    g_o = g_d * 0.5 * (1.0 - t * t)      # dd/do
    gW3 = g_o.T @ a2
    gb3 = g_o.sum(axis=0)
    g_a2 = g_o @ W3
    g_z2 = g_a2 * (1.0 - a2 * a2)
    gW2 = g_z2.T @ a1
    gb2 = g_z2.sum(axis=0)
    g_a1 = g_z2 @ W2
    g_z1 = g_a1 * (1.0 - a1 * a1)
    gW1 = g_z1.T @ X
    gb1 = g_z1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ training data

def leaf_stats(x, y, perm, begin, end):
    """S (L x 9) = [S_xy | S_yy | S_xx] per leaf and component, summed over the rows of
    x and y (nrhs x 3N, user order)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    L = len(begin)
    S = np.zeros((L, 9))
    for l in range(L):
        idx = perm[begin[l]:end[l]]
        for a in range(3):
            dofs = 3 * idx + a
            xa, ya = x[:, dofs], y[:, dofs]
            S[l, a] = float((xa * ya).sum())
            S[l, 3 + a] = float((ya * ya).sum())
            S[l, 6 + a] = float((xa * xa).sum())
    return S


def samples(S_list):
    """Normalised training targets Q for a list of per-system stats."""
    ns = len(S_list)
    out = []
    for S in S_list:
        T = S[:, 6:9].sum()
        out.append(S / (ns * T))
    return np.vstack(out)


def apply(d, r, perm, begin, end, binv_apply):
    """z = D B^-1 r (user order), binv_apply the block-Jacobi inverse."""
    z = binv_apply(r)
    for l in range(len(begin)):
        idx = perm[begin[l]:end[l]]
        for a in range(3):
            z[3 * idx + a] *= d[l, a]
    return z


# ------------------------------------------------------------------ near correction
# The second kind of correction: M^-1 r = y - gamma D B^-1 N y, y = B^-1 r, N the
# near-field blocks of E off the diagonal leaf blocks.  Trained on the fit of D w to
# y - x (w = B^-1 N y): the same loss as above with x' = y - x and y' = w.

def near_offdiag(Emat, tree, eta=2.0):
    """N (3N x 3N, user order): the entries of E in the inadmissible leaf pairs of the
    block partition, minus the diagonal leaf blocks."""
    from . import oracle as O
    n = Emat.shape[0]
    Nm = np.zeros((n, n))
    near, _ = O.block_partition(tree, eta)
    for s, t in near:
        if s == t:
            continue
        rs = O.dof_index(tree.perm[tree.begin[s]:tree.end[s]])
        ct = O.dof_index(tree.perm[tree.begin[t]:tree.end[t]])
        Nm[np.ix_(rs, ct)] = Emat[np.ix_(rs, ct)]
    return Nm


def near_stats(x, b, Nm, perm, begin, end, binv_apply):
    """Per (leaf, component) statistics of (y - x, w), y = B^-1 b, w = B^-1 N y."""
    bb = np.atleast_2d(b)
    y = np.vstack([binv_apply(v) for v in bb])
    w = np.vstack([binv_apply(Nm @ v) for v in y])
    return leaf_stats(y - np.atleast_2d(x), w, perm, begin, end)


def apply_near(d, gamma, r, Nm, perm, begin, end, binv_apply):
    """z = y - gamma D B^-1 N y, y = B^-1 r (user order)."""
    y = binv_apply(r)
    u = binv_apply(Nm @ y)
    z = y.copy()
    for l in range(len(begin)):
        idx = perm[begin[l]:end[l]]
        for a in range(3):
            z[3 * idx + a] -= gamma * d[l, a] * u[3 * idx + a]
    return z
