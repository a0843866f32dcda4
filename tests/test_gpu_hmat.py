"""GPU parity of the assembled H-matrix and its product against the CPU FP64 oracle,
through the C-ABI.

Bar (the accuracy the method promises): for FP32 factors the product matches the dense
oracle product E x to a relative L2 error of eps + 1e-6; every compressed block
satisfies ||U V^T - E_st||_F <= kappa eps ||E_st||_F with kappa the truncation factor
(recompression to kappa eps / 2, the cross approximation to kappa eps / 10 per step, a
heuristic stop); the F64 product applies the stored operator, so its distance to the
dense product is bounded by the same eps + 1e-6.  BF16 factors are stated, not hidden:
relative error below 1e-2.
Sizes span many leaves with ragged leaf sizes (N not a power of two), both cluster
orders and the full 51,468-element fault on sampled receiver rows."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import hmat, synth

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.25


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def build_h(el, leaf, eps, storage="f32", eta=2.0):
    T = hmat.ClusterTree(el, leaf, eta)
    H = hmat.HMatrix(T, el, E, NU, eps, storage)
    return T, H


def run_mv(dev, H, x_np, dtype):
    import torch
    x = torch.as_tensor(x_np, dtype=dtype, device=dev).contiguous()
    y = torch.empty_like(x)
    H.matvec(x, y)
    H.check()
    return y.cpu().numpy().astype(np.float64)


CASES = [("penny40", lambda: synth.config_penny(40), 64, 1e-6),
         ("planes16", lambda: synth.config_three_planes(16), 32, 1e-6),
         ("crackfault", lambda: synth.config_crack_fault(h=0.08), 48, 1e-5)]


@pytest.mark.parametrize("name,mk,leaf,eps", CASES)
def test_matvec_matches_dense_oracle(dev, name, mk, leaf, eps):
    import torch
    el = mk()
    T, H = build_h(el, leaf, eps)
    A = O.dense_matrix(el, E, NU)
    X = synth.rhs_normal(3 * el.N, 5, nrhs=3)
    for k in range(3):
        ref = A @ X[k]
        y32 = run_mv(dev, H, X[k], torch.float32)
        y64 = run_mv(dev, H, X[k], torch.float64)
        assert rel(y32, ref) <= eps + 1e-6, (name, rel(y32, ref))
        assert rel(y64, ref) <= eps + 1e-6, (name, rel(y64, ref))
    # physical right-hand side as well
    b = synth.rhs_uniform_pressure(el)
    assert rel(run_mv(dev, H, b, torch.float64), A @ b) <= eps + 1e-6


@pytest.mark.parametrize("eps,kappa", [(1e-6, 1.0), (1e-6, 0.0), (1e-4, 0.0)])
def test_aca_blocks_meet_tolerance(dev, eps, kappa):
    """Every compressed block meets its per-block accuracy trunc_factor * eps (the
    library default, 30, for kappa = 0)."""
    el = synth.config_three_planes(24)
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "f32", trunc_factor=kappa)
    tol = (kappa if kappa > 0 else 30.0) * eps
    ex = T.export()
    perm, begin, end = ex["perm"], ex["begin"], ex["end"]
    far = ex["far"]
    rng = np.random.default_rng(0)
    checked = 0
    for b in rng.choice(len(far), size=min(120, len(far)), replace=False):
        s, t = far[b]
        rs = perm[begin[s]:end[s]]
        rt = perm[begin[t]:end[t]]
        f = H.far_factor_arrays(b, len(rs), len(rt))
        if f is None:  # kept dense: its factors would not be smaller
            continue
        U, V = f
        Ed = O.dense_rows(el, E, NU, rs)[:, O.dof_index(rt)]
        assert np.linalg.norm(U @ V.T - Ed) <= tol * np.linalg.norm(Ed), b
        # recompressed factors: V has orthonormal columns
        assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-5)
        checked += 1
    assert checked >= 20


def test_f64_product_is_consistent_with_f32_storage(dev):
    import torch
    el = synth.config_penny(40)
    T, H = build_h(el, 64, 1e-6)
    x = synth.rhs_normal(3 * el.N, 6)
    y64 = run_mv(dev, H, x, torch.float64)
    y32 = run_mv(dev, H, x, torch.float32)
    # same stored operator: differ only by FP32 rounding of x and of the accumulation
    assert rel(y32, y64) < 2e-6
    # linearity at FP64 accuracy of the stored operator
    x2 = synth.rhs_normal(3 * el.N, 7)
    ya = run_mv(dev, H, x + 0.5 * x2, torch.float64)
    yb = y64 + 0.5 * run_mv(dev, H, x2, torch.float64)
    assert rel(ya, yb) < 1e-11


def test_bf16_factors_error_is_stated(dev):
    import torch
    el = synth.config_three_planes(16)
    T, H = build_h(el, 32, 1e-6, "bf16")
    A = O.dense_matrix(el, E, NU)
    x = synth.rhs_normal(3 * el.N, 8)
    e = rel(run_mv(dev, H, x, torch.float64), A @ x)
    assert e < 1e-2
    print("BF16 factors: relative error %.2e" % e)


@pytest.mark.parametrize("name,mk,leaf", [("penny40", lambda: synth.config_penny(40), 64),
                                          ("planes16", lambda: synth.config_three_planes(16), 32)])
def test_bf16_single_rhs_tensor_core_phase(dev, name, mk, leaf):
    """BF16 factors with one RHS apply the U slices of phase 2 on tensor cores (t split
    into BF16 hi + lo, about 16 bits kept).  The FP32 product agrees with the F64 product
    of the same stored operator (CUDA cores, compensated) to 2e-5 -- the split, not the
    BF16 factors, sets this bar -- and with the dense oracle to the BF16 bound."""
    import torch
    el = mk()
    T, H = build_h(el, leaf, 1e-6, "bf16")
    x = synth.rhs_normal(3 * el.N, 62)
    y32 = run_mv(dev, H, x, torch.float32)
    y64 = run_mv(dev, H, x, torch.float64)
    assert rel(y32, y64) < 2e-5, (name, rel(y32, y64))
    assert rel(y32, O.dense_matrix(el, E, NU) @ x) < 1e-2
    print("%s: BF16 FP32 vs F64 product %.2e" % (name, rel(y32, y64)))


def test_factor_stream_layouts(dev):
    """FP32 factor streams pad each leaf slice to a multiple of 8 rows; the BF16 copies pad
    further to an odd number of 16-byte lines (8 more rows where the FP32 stride has an even
    count), with their own offsets.  The stored bytes of an FP32 and of a BF16 H-matrix of
    one tree then leave the same near-field bytes once the factor entries of both layouts,
    counted here from the leaves and the block ranks, are taken off."""
    el = synth.config_three_planes(16)
    T = hmat.ClusterTree(el, 32, 2.0)
    H32 = hmat.HMatrix(T, el, E, NU, 1e-6, "f32")
    H16 = hmat.HMatrix(T, el, E, NU, 1e-6, "bf16")
    ex = T.export()
    begin, end, left = ex["begin"], ex["end"], ex["left"]
    leaves = [q for q in range(len(left)) if left[q] < 0]
    ld = {q: -(-3 * (end[q] - begin[q]) // 8) * 8 for q in leaves}
    ld16 = {q: ld[q] if (ld[q] // 8) % 2 == 1 else ld[q] + 8 for q in leaves}
    assert all((v // 8) % 2 == 1 and v % 8 == 0 for v in ld16.values())

    def padded_rows(node, table):
        return sum(table[q] for q in leaves if begin[node] <= begin[q] < end[node])

    def factor_entries(H, table):
        tot = 0
        for b, (s, t) in enumerate(ex["far"]):
            r = H.far_factors(b)
            if r > 0:
                tot += r * (padded_rows(s, table) + padded_rows(t, table))
        return tot

    for H in (H32, H16):
        assert H.info()["n_far_refined"] == 0
    near32 = H32.info()["stored_bytes"] - 4 * factor_entries(H32, ld)
    near16 = H16.info()["stored_bytes"] - 2 * factor_entries(H16, ld16)
    assert near32 == near16 and near32 > 0


def test_multi_rhs_equals_columns(dev):
    import torch
    el = synth.config_three_planes(16)
    T, H = build_h(el, 32, 1e-6)
    X = synth.rhs_normal(3 * el.N, 9, nrhs=5)
    Y = run_mv(dev, H, X, torch.float64)
    for k in range(5):
        assert rel(Y[k], run_mv(dev, H, X[k], torch.float64)) < 1e-12


def test_repeated_products_are_bitwise_identical(dev):
    import torch
    el = synth.config_penny(40)
    T, H = build_h(el, 32, 1e-6)
    x = synth.rhs_normal(3 * el.N, 10)
    ys = [run_mv(dev, H, x, torch.float32) for _ in range(3)]
    assert all(np.array_equal(ys[0], y) for y in ys[1:])


def test_full_size_fault_sampled_rows(dev):
    """51,468-element fault (leaf 64, eta 2, eps 1e-6) on 300 seeded receiver rows."""
    import torch
    el = synth.config_fault(256)
    eps = 1e-6
    T, H = build_h(el, 64, eps)
    x = synth.rhs_shear_plus_bump(el)
    y = run_mv(dev, H, x, torch.float64)
    rng = np.random.default_rng(1603)
    rows = np.sort(rng.choice(el.N, size=300, replace=False))
    ref = O.dense_matvec_rows(el, E, NU, x, rows)
    got = y.reshape(-1, 3)[rows].ravel()
    assert rel(got, ref) <= eps + 1e-6
    info = H.info()
    assert info["rank_max"] <= 160 and info["near_entries"] > 0


@pytest.mark.parametrize("max_rank,eps", [(6, 1e-6), (12, 1e-4)])
def test_blocks_over_the_rank_cap_are_refined(dev, max_rank, eps):
    """A rank cap too small for the tolerance: non-converging admissible blocks are
    replaced by their children's blocks (down to dense leaf pairs) and the product still
    meets eps + 1e-6 against the dense oracle."""
    import torch
    el = synth.config_three_planes(24)
    T = hmat.ClusterTree(el, 16, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "f32", max_rank=max_rank)
    info = H.info()
    nfar = T.info()["n_far"]
    assert info["n_far_refined"] > 0 and info["rank_max"] <= max_rank
    ranks = [H.far_factors(b) for b in range(nfar)]
    assert sum(r == -2 for r in ranks) > 0
    A = O.dense_matrix(el, E, NU)
    x = synth.rhs_normal(3 * el.N, 41)
    assert rel(run_mv(dev, H, x, torch.float32), A @ x) <= eps + 1e-6
    assert rel(run_mv(dev, H, x, torch.float64), A @ x) <= eps + 1e-6


@pytest.mark.parametrize("nrhs", [16, 13])
def test_bf16_multi_rhs_tensor_core_phase(dev, nrhs):
    """BF16 factors with 16 RHS run phase 1 on tensor cores (x split into BF16 hi + lo,
    about 16 bits kept); 13 RHS take the CUDA-core path.  Both agree with the single-RHS
    products to 1e-4 (the x split, relative to the whole product) and with the dense
    oracle to the BF16 bound."""
    import torch
    el = synth.config_three_planes(16)
    T, H = build_h(el, 32, 1e-6, "bf16")
    X = synth.rhs_normal(3 * el.N, 51, nrhs=nrhs)
    Y = run_mv(dev, H, X, torch.float32)
    A = O.dense_matrix(el, E, NU)
    for q in range(nrhs):
        yq = run_mv(dev, H, X[q], torch.float32)
        assert rel(Y[q], yq) < 1e-4, q
        assert rel(Y[q], A @ X[q]) < 1e-2


def test_factor_precision_choice(dev):
    """With both precisions stored, hm_matvec_factors picks either; the BF16 choice equals
    the product of an H-matrix that stores BF16 only (same assembly, same plan); asking for
    a precision that is not stored is an error."""
    import torch
    el = synth.config_penny(24)
    T = hmat.ClusterTree(el, 32, 2.0)
    Hb = hmat.HMatrix(T, el, E, NU, 1e-6, "both")
    H16 = hmat.HMatrix(T, el, E, NU, 1e-6, "bf16")
    H32 = hmat.HMatrix(T, el, E, NU, 1e-6, "f32")
    x = torch.as_tensor(synth.rhs_normal(3 * el.N, 61), dtype=torch.float32, device=dev)
    outs = {}
    for name, H, fac in (("both16", Hb, "bf16"), ("only16", H16, None), ("both32", Hb, "f32"), ("only32", H32, None)):
        y = torch.empty_like(x)
        H.matvec(x, y, factors=fac)
        outs[name] = y
    torch.cuda.synchronize()
    assert torch.equal(outs["both16"], outs["only16"]) and torch.equal(outs["both32"], outs["only32"])
    with pytest.raises(hmat.HMError) as ei:
        H16.matvec(x, torch.empty_like(x), factors="f32")
    assert ei.value.status == hmat.HM_EINVAL


@pytest.mark.parametrize("n_grid,leaf", [(12, 16), (24, 32), (24, 64)])
def test_small_operators_with_fewer_chunks_than_ctas(dev, n_grid, leaf):
    """Operators whose coefficient streams hold about as many chunks as there are SMs (or
    fewer): chunks larger than a per-CTA byte share once left CTAs without a chunk inside
    a row leaf split over several CTAs, whose result was then never written.  Products
    match the dense oracle and repeat bit for bit (the split-leaf arrival counters are
    left clean), for both factor precisions."""
    import torch
    el = synth.config_penny(n_grid)
    T = hmat.ClusterTree(el, leaf, 2.0)
    H = hmat.HMatrix(T, el, E, NU, 1e-6, "both")
    A = O.dense_matrix(el, E, NU)
    x = synth.rhs_normal(3 * el.N, 63)
    ref = A @ x
    for fac, bar in (("f32", 1e-6 + 1e-6), ("bf16", 1e-6 + 2.0 ** -8)):
        xt = torch.as_tensor(x, dtype=torch.float32, device=dev)
        ys = []
        for _ in range(3):
            y = torch.full_like(xt, float("nan"))
            H.matvec(xt, y, factors=fac)
            H.check()
            ys.append(y.cpu().numpy().astype(np.float64))
        assert all(np.array_equal(ys[0], y) for y in ys[1:]), fac
        assert rel(ys[0], ref) <= bar, (fac, rel(ys[0], ref))


def test_a_withheld_copy_times_out_and_the_operator_stays_usable(dev):
    """Failure path of the copy pipeline, with no fault: the test switch of
    hm_hmat_set_wait makes the row phase's producer withhold a chunk, the consumers'
    1 ms waits run out, hm_hmat_check reports HM_ETIMEOUT (and clears the flags and
    counters); with the switch off the next products are correct again."""
    import torch
    el = synth.config_penny(16)
    T, H = build_h(el, 16, 1e-6)
    A = O.dense_matrix(el, E, NU)
    x = synth.rhs_normal(3 * el.N, 64)
    xt = torch.as_tensor(x, dtype=torch.float32, device=dev)
    for chunk in (0, 3):
        H.set_wait(1e-3, chunk)
        y = torch.empty_like(xt)
        H.matvec(xt, y)
        with pytest.raises(hmat.HMError) as ei:
            H.check()
        assert ei.value.status == hmat.HM_ETIMEOUT
        H.set_wait(2.0, -1)
        assert rel(run_mv(dev, H, x, torch.float32), A @ x) <= 1e-6 + 1e-6
