"""Parity of the exact product paths the solvers and the benchmark serve, through the C-ABI.

Two kinds of check:

* Element by element against the stored operator.  The H-matrix is exported (the FP32
  factors of every admissible block; near blocks from the oracle, rounded to FP32 as the
  library stores them) and rebuilt in numpy FP64 -- with the factors rounded to BF16
  (round to nearest even) for the BF16 paths.  Every output entry of every path must
  match that product to 1e-5 of the row's absolute scale
  s_i = sum_j |A_ij| |x_j| + sum_b sum_k |U_ik| |(V^T x)_k|  (FP32 vectors: FP32
  accumulation and, on the tensor-core paths, the vector split into BF16 hi + lo, about
  16 bits) or to 2e-7 of it (FP64 vectors: compensated products; the near entries the
  library evaluates in FP64 and the oracle's may round to FP32 one ulp apart, at most
  2^-23 of each term).  A dropped,
  duplicated or misplaced slice of any block moves whole entries and fails this, where a
  norm bar of 1e-2 would not.
* Against the FP64 oracle on 300 seeded receiver rows at full size: the 51,468-element
  fault (the compensated FP64 product; F32 vectors with FP32 factors; F32 vectors with
  BF16 factors and one right-hand side -- the inner product of the mixed solver) and
  three intersecting 190 x 190 planes (108,300 elements) with 16 right-hand sides (the
  BF16 tensor-core V^T x contraction and the FP32 16-RHS product).  Bars, with y the
  exact product of the sampled rows and s = |E| |x| their absolute sums:
    FP64 vectors:  ||y_H - y|| <= (eps + 1e-6) ||y||  (the ACA accuracy);
    FP32 vectors:  ||y_H - y|| <= (eps + 1e-6) ||y|| + 1e-6 ||s||  -- FP32 rounding of a
      sum is bounded relative to the sum of the magnitudes, not to the result, and the
      fault's right-hand side (uniform slip plus a bump) cancels: ||s|| / ||y|| is
      printed;
    BF16 factors:  the FP32 bar with eps + 2^-8 in place of eps: each stored factor
      entry carries a relative rounding error of at most 2^-9, so each term U_ik V_jk
      of a block is off by at most about 2^-8 of itself.
  Each measured error is printed.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import hmat, synth

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.25
BF16_BOUND = 2.0 ** -8


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def bf16_round(a):
    """FP32 -> BF16 -> FP64, round to nearest even (the library's storage rounding)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def stored_operator(el, T, H, bf16):
    """Dense FP64 copy of the stored H-matrix (user DOF order) and its low-rank blocks."""
    A = O.dense_matrix(el, E, NU).astype(np.float32).astype(np.float64)
    ex = T.export()
    perm, begin, end = ex["perm"], ex["begin"], ex["end"]
    assert H.info()["n_far_refined"] == 0
    blocks = []
    for b, (s, t) in enumerate(ex["far"]):
        rs, rt = perm[begin[s]:end[s]], perm[begin[t]:end[t]]
        f = H.far_factor_arrays(b, len(rs), len(rt))
        if f is None:  # stored dense: FP32 tiles of the near stream
            continue
        U, V = f
        if bf16:
            U, V = bf16_round(U), bf16_round(V)
        di, dj = O.dof_index(rs), O.dof_index(rt)
        A[np.ix_(di, dj)] = U @ V.T
        blocks.append((di, dj, U, V))
    return A, blocks


def row_scale(A, blocks, x):
    s = np.abs(A) @ np.abs(x)
    for di, dj, U, V in blocks:
        s[di] += np.abs(U) @ np.abs(V.T @ x[dj])
    return s


def product(dev, H, X, dtype, factors):
    import torch
    x = torch.as_tensor(X, dtype=dtype, device=dev).contiguous()
    y = torch.empty_like(x)
    H.matvec(x, y, factors=factors)
    H.check()
    return y.cpu().numpy().astype(np.float64)


def worst(y, ref, scale):
    return float(np.max(np.abs(y - ref) / scale))


SMALL = [("penny40", lambda: synth.config_penny(40), 64, 1e-6),
         ("planes16", lambda: synth.config_three_planes(16), 32, 1e-6),
         ("crackfault", lambda: synth.config_crack_fault(h=0.1), 48, 1e-5)]


@pytest.mark.parametrize("name,mk,leaf,eps", SMALL)
def test_every_path_entrywise_against_the_stored_operator(dev, name, mk, leaf, eps):
    import torch
    el = mk()
    T = hmat.ClusterTree(el, leaf, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "both")
    ops = {fac: stored_operator(el, T, H, fac == "bf16") for fac in ("f32", "bf16")}
    X = synth.rhs_normal(3 * el.N, 71, nrhs=16)
    X32 = X.astype(np.float32).astype(np.float64)
    report = []
    for fac in ("f32", "bf16"):
        A, blocks = ops[fac]
        # one right-hand side, FP32 vectors (BF16: the U slices on tensor cores) and FP64 vectors
        for q in range(2):
            ref32 = A @ X32[q]
            e = worst(product(dev, H, X32[q], torch.float32, fac), ref32, row_scale(A, blocks, X32[q]))
            assert e <= 1e-5, (name, fac, "f32 vectors", q, e)
            ref64 = A @ X[q]
            e64 = worst(product(dev, H, X[q], torch.float64, fac), ref64, row_scale(A, blocks, X[q]))
            assert e64 <= 2e-7, (name, fac, "f64 vectors", q, e64)
            report.append((fac, 1, e, e64))
        # 16 right-hand sides (BF16: V^T x on tensor cores) and 3 (CUDA cores)
        for nr in (16, 3):
            Y = product(dev, H, X32[:nr], torch.float32, fac)
            e = max(worst(Y[q], A @ X32[q], row_scale(A, blocks, X32[q])) for q in range(nr))
            assert e <= 1e-5, (name, fac, nr, e)
            report.append((fac, nr, e, None))
    for fac, nr, e, e64 in report:
        print("%s %s factors, %2d RHS: worst entry / row scale %.2e (f32 vectors)%s" % (
            name, fac, nr, e, "" if e64 is None else ", %.2e (f64 vectors)" % e64))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_rows_and_scale(el, X, rows, chunk=25):
    """Exact products of the sampled receiver rows and their absolute sums |E| |x|, for
    each right-hand side in X (nrhs x 3N), from the oracle's dense rows."""
    X = np.atleast_2d(X)
    Y = np.empty((X.shape[0], 3 * rows.size))
    S = np.empty_like(Y)
    for c0 in range(0, rows.size, chunk):
        R = O.dense_rows(el, E, NU, rows[c0:c0 + chunk])
        Y[:, 3 * c0:3 * c0 + R.shape[0]] = (R @ X.T).T
        S[:, 3 * c0:3 * c0 + R.shape[0]] = (np.abs(R) @ np.abs(X).T).T
    return Y, S


def test_full_size_fault_served_products(dev):
    """The 51,468-element fault (leaf 64, eta 2, eps 1e-6) on 300 seeded receiver rows:
    the compensated FP64 product, the FP32 product with FP32 factors and the mixed
    solver's inner product (FP32 vectors, BF16 factors, one RHS)."""
    import torch
    el = synth.config_fault(256)
    eps = 1e-6
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "both")
    x = synth.rhs_shear_plus_bump(el)
    x32 = x.astype(np.float32).astype(np.float64)
    rows = np.sort(np.random.default_rng(1603).choice(el.N, size=300, replace=False))
    ref, S = oracle_rows_and_scale(el, np.stack([x, x32]), rows)
    # the matrix-free oracle product agrees with the stored oracle rows
    assert rel(O.dense_matvec_rows(el, E, NU, x, rows), ref[0]) < 1e-13

    def pick(y):
        return y.reshape(-1, 3)[rows].ravel()

    y64 = pick(product(dev, H, x, torch.float64, "f32"))
    y32 = pick(product(dev, H, x32, torch.float32, "f32"))
    y16 = pick(product(dev, H, x32, torch.float32, "bf16"))
    cond = float(np.linalg.norm(S[1]) / np.linalg.norm(ref[1]))
    print("51,468-element fault, shear + bump: ||E||x|| / ||E x|| = %.1f on 300 rows" % cond)
    for name, y, r in (("f64 vectors, f32 factors", y64, ref[0]), ("f32 vectors, f32 factors", y32, ref[1]),
                       ("f32 vectors, bf16 factors", y16, ref[1])):
        print("51,468-element fault, %s: relative L2 error %.3e on 300 rows" % (name, rel(y, r)))
    assert rel(y64, ref[0]) <= eps + 1e-6
    n_ref, n_s = np.linalg.norm(ref[1]), np.linalg.norm(S[1])
    assert np.linalg.norm(y32 - ref[1]) <= (eps + 1e-6) * n_ref + 1e-6 * n_s
    assert np.linalg.norm(y16 - ref[1]) <= (eps + BF16_BOUND) * n_ref + 1e-6 * n_s


def test_three_planes_16_rhs_served_products(dev):
    """Three intersecting 190 x 190 planes (N = 108,300; leaf 64, eta 2, eps 1e-5),
    16 seeded N(0, 1) right-hand sides in one product: BF16 factors (V^T x on the tensor
    cores) and FP32 factors, against the oracle on 300 receiver rows for every RHS."""
    import torch
    el = synth.config_three_planes(190)
    assert el.N == 108300
    eps = 1e-5
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "both")
    X32 = synth.rhs_normal(3 * el.N, 1603, nrhs=16).astype(np.float32).astype(np.float64)
    rows = np.sort(np.random.default_rng(1606).choice(el.N, size=300, replace=False))
    ref, S = oracle_rows_and_scale(el, X32, rows)
    pick = (3 * rows[:, None] + np.arange(3)).ravel()
    for fac, e_op in (("f32", eps), ("bf16", eps + BF16_BOUND)):
        Y = product(dev, H, X32, torch.float32, fac)
        e = [rel(Y[q][pick], ref[q]) for q in range(16)]
        print("three planes N=108,300, %s factors, 16 RHS: relative L2 error max %.3e, mean %.3e on 300 rows" % (
            fac, max(e), float(np.mean(e))))
        for q in range(16):
            bar = (e_op + 1e-6) * np.linalg.norm(ref[q]) + 1e-6 * np.linalg.norm(S[q])
            assert np.linalg.norm(Y[q][pick] - ref[q]) <= bar, (fac, q, e[q])
