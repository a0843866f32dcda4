"""GPU parity of the batch of independent faults (block-diagonal operator in one arena),
the graph-replayed product and the leaf-size autotuner, through the C-ABI.

Bar: the batch product matches, fault by fault, the oracle's dense product of that
fault's own operator (its own nu) to eps + 1e-6 relative L2, like a single H-matrix;
against the products of the separately assembled parts it differs only by FP32
summation order (1e-6).  The block-diagonal solve agrees with per-fault solves and with
the oracle's dense LU per fault.  A graph replay computes exactly the same numbers as
the eager product (same plan, same deterministic order: bitwise equal)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import hmat, synth

pytestmark = pytest.mark.gpu

E = 1.0


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


@pytest.fixture(scope="module")
def faults(dev):
    """Four disk faults of 300-1500 elements, seeded normals and nu in [0.2, 0.3]."""
    els, nus = synth.config_faults_batch(n_faults=4, seed=1604, n_min=300, n_max=1500)
    return els, nus


def assemble_parts(els, nus, eps, storage="f32", leaf=32):
    trees, parts = [], []
    for el, nu in zip(els, nus):
        T = hmat.ClusterTree(el, leaf, 2.0)
        trees.append(T)
        parts.append(hmat.HMatrix(T, el, E, float(nu), eps, storage))
    return trees, parts


def test_batch_product_matches_dense_oracle_per_fault(dev, faults):
    import torch
    els, nus = faults
    eps = 1e-6
    trees, parts = assemble_parts(els, nus, eps)
    B = hmat.HMatrix.batch(parts)
    n = [3 * el.N for el in els]
    assert B.info()["n_dof"] == sum(n)
    x = synth.random_vector(sum(n), 5)
    xt = torch.as_tensor(x, dtype=torch.float32, device=dev)
    yt = torch.empty_like(xt)
    B.matvec(xt, yt)
    B.check()
    y = yt.cpu().numpy().astype(np.float64)
    off = 0
    for el, nu, H, nf in zip(els, nus, parts, n):
        ref = O.dense_matrix(el, E, float(nu)) @ x[off:off + nf]
        assert rel(y[off:off + nf], ref) < eps + 1e-6
        # the separately assembled part gives the same product up to summation order
        xp = xt[off:off + nf].clone()
        yp = torch.empty_like(xp)
        H.matvec(xp, yp)
        assert rel(y[off:off + nf], yp.cpu().numpy().astype(np.float64)) < 1e-6
        off += nf


def test_batch_info_adds_up(dev, faults):
    els, nus = faults
    trees, parts = assemble_parts(els, nus, 1e-6)
    B = hmat.HMatrix.batch(parts)
    bi = B.info()
    infos = [p.info() for p in parts]
    for k in ("n_dof", "near_entries", "far_entries", "u_entries", "v_entries", "tb_len", "p_len", "n_far_lowrank",
              "n_far_dense"):
        assert bi[k] == sum(i[k] for i in infos), k
    assert bi["rank_max"] == max(i["rank_max"] for i in infos)


def test_batch_f64_multi_rhs_and_bf16(dev, faults):
    import torch
    els, nus = faults
    trees, parts = assemble_parts(els[:2], nus[:2], 1e-6, storage="both")
    B = hmat.HMatrix.batch(parts)
    n = [3 * el.N for el in els[:2]]
    X = synth.rhs_normal(sum(n), 21, nrhs=3)
    xt = torch.as_tensor(X, dtype=torch.float64, device=dev).contiguous()
    yt = torch.empty_like(xt)
    B.matvec(xt, yt)
    B.check()
    Y = yt.cpu().numpy()
    off = 0
    for el, nu, nf in zip(els[:2], nus[:2], n):
        A = O.dense_matrix(el, E, float(nu))
        for q in range(3):
            assert rel(Y[q, off:off + nf], A @ X[q, off:off + nf]) < 2e-6
        off += nf


def test_block_diagonal_solve_matches_per_fault(dev, faults):
    import torch
    els, nus = faults
    trees, parts = assemble_parts(els[:3], nus[:3], 1e-9, storage="both")
    B = hmat.HMatrix.batch(parts)
    n = [3 * el.N for el in els[:3]]
    rng = np.random.default_rng(3)
    h = 2.0 / 256
    ks = [np.exp(rng.uniform(math.log(1e-3), math.log(1e2), size=el.N)) * (E / h) for el in els[:3]]
    b = synth.rhs_normal(sum(n), 22)
    bt = torch.as_tensor(b, device=dev)
    for mode in ("f64", "mixed"):
        xt = torch.zeros_like(bt)
        info = B.solve(bt, xt, torch.as_tensor(np.concatenate(ks), device=dev), mode=mode)
        assert info[0]["relres"] <= 1e-8
        x = xt.cpu().numpy()
        off = 0
        for el, nu, H, k, nf in zip(els[:3], nus[:3], parts, ks, n):
            A = O.tangent_dense(O.dense_matrix(el, E, float(nu)), k, 0.0)
            x_lu = np.linalg.solve(A, b[off:off + nf])
            assert rel(x[off:off + nf], x_lu) < 1e-6
            off += nf


def test_graph_replay_is_bitwise_equal(dev, faults):
    import torch
    els, nus = faults
    trees, parts = assemble_parts(els, nus, 1e-6)
    B = hmat.HMatrix.batch(parts)
    nd = B.info()["n_dof"]
    for dt in (torch.float32, torch.float64):
        x = torch.as_tensor(synth.random_vector(nd, 31), dtype=dt, device=dev)
        y0 = torch.empty_like(x)
        y1 = torch.empty_like(x)
        B.matvec(x, y0)
        B.matvec_graph(x, y1)  # eager run + capture + first replay
        torch.cuda.synchronize()
        assert torch.equal(y0, y1)
        # new data in the same buffers: the replay reads them
        x.copy_(torch.as_tensor(synth.random_vector(nd, 32), dtype=dt, device=dev))
        B.matvec(x, y0)
        for _ in range(3):
            B.matvec_graph(x, y1)
        B.check()
        assert torch.equal(y0, y1)
    # timing on: plain product, same numbers
    B.timing(True)
    B.matvec_graph(x, y1)
    B.timing(False)
    assert B.timing_read()["count"] == 1
    assert torch.equal(y0, y1)


def test_graph_replay_several_rhs(dev, faults):
    import torch
    els, nus = faults
    T = hmat.ClusterTree(els[0], 32, 2.0)
    H = hmat.HMatrix(T, els[0], E, float(nus[0]), 1e-6)
    X = torch.as_tensor(synth.rhs_normal(3 * els[0].N, 33, nrhs=4), dtype=torch.float32, device=dev)
    Y0, Y1 = torch.empty_like(X), torch.empty_like(X)
    H.matvec(X, Y0)
    H.matvec_graph(X, Y1)
    H.matvec_graph(X, Y1)
    H.check()
    assert torch.equal(Y0, Y1)


def test_autotune_picks_fastest_and_caches(dev, faults, tmp_path):
    els, nus = faults
    el = els[-1]
    cache = str(tmp_path / "tune.json")
    res = hmat.autotune(el, E, float(nus[-1]), 1e-6, "f32", leaves=(16, 32, 64), etas=(2.0,), budget_ms=600000,
                        cache=cache)
    cands = res["candidates"]
    assert res["tuned"] == 3 and [c["leaf"] for c in cands] == [16, 32, 64]
    best = min(cands, key=lambda c: c["ms"])
    assert res["best"]["leaf"] == best["leaf"] and all(c["ms"] > 0 for c in cands)
    with open(cache) as f:
        table = json.load(f)
    assert len(table) == 1
    again = hmat.autotune(el, E, float(nus[-1]), 1e-6, "f32", leaves=(16, 32, 64), etas=(2.0,), cache=cache)
    assert again == res
    # a budget of 0 ms still times the first candidate, and only it
    one = hmat.autotune(el, E, float(nus[-1]), 1e-6, "f32", leaves=(16, 32), etas=(2.0,), budget_ms=0)
    assert one["tuned"] == 1 and one["best"]["leaf"] == 16
    os.remove(cache)


def test_tile_shapes_give_the_same_product(dev, faults):
    """Every tile shape the autotuner may choose (chunk bytes and columns, ring depth,
    consumer warps) computes the batch product of the default shape to FP32 summation
    order (the chunks, hence the order of the partial sums, change), for FP32 and BF16
    factors and one and three right-hand sides; a shape outside the ranges is refused."""
    import torch
    els, nus = faults
    trees, parts = assemble_parts(els, nus, 1e-6, storage="both")
    B = hmat.HMatrix.batch(parts)
    x = torch.as_tensor(synth.rhs_normal(B.ndof, 71, nrhs=3), dtype=torch.float32, device=dev)
    ref = {}
    for fac in ("f32", "bf16"):
        for nr in (1, 3):
            y = torch.empty_like(x[:nr])
            B.matvec(x[:nr].contiguous(), y, factors=fac)
            ref[fac, nr] = y.cpu().numpy().astype(np.float64)
    for shape in hmat.DEFAULT_SHAPES[1:]:
        B.set_tile_shape(shape)
        assert B.tile_shape() == tuple(shape)
        for fac in ("f32", "bf16"):
            for nr in (1, 3):
                y = torch.empty_like(x[:nr])
                B.matvec(x[:nr].contiguous(), y, factors=fac)
                B.check()
                got = y.cpu().numpy().astype(np.float64)
                assert rel(got, ref[fac, nr]) < 2e-6, (shape, fac, nr, rel(got, ref[fac, nr]))
    with pytest.raises(hmat.HMError) as ei:
        B.set_tile_shape((32768, 128, 5, 16))
    assert ei.value.status == hmat.HM_EINVAL


def test_tile_shape_tuning_keeps_the_fastest(dev, faults):
    """hm_tune_tile_shape times every candidate and leaves the fastest on the H-matrix;
    the autotuner searches shapes together with the leaf size."""
    els, nus = faults
    trees, parts = assemble_parts(els, nus, 1e-6)
    B = hmat.HMatrix.batch(parts)
    res = B.tune_tile_shape(reps=10)
    cands = res["candidates"]
    assert res["tuned"] == len(hmat.DEFAULT_SHAPES) == len(cands)
    best = min(cands, key=lambda c: c["ms"])
    assert res["best"]["ms"] == best["ms"]
    key = (best["chunk_bytes"], best["chunk_cols"], best["ring"], best["warps"])
    assert B.tile_shape() == key
    at = hmat.autotune(els[-1], E, float(nus[-1]), 1e-6, "f32", leaves=(16, 32), etas=(2.0,), budget_ms=600000,
                       shapes=hmat.DEFAULT_SHAPES[:3])
    assert at["tuned"] == 6
    b = min(at["candidates"], key=lambda c: c["ms"])
    assert (at["best"]["leaf"], at["best"]["chunk_bytes"], at["best"]["chunk_cols"]) == (
        b["leaf"], b["chunk_bytes"], b["chunk_cols"])
