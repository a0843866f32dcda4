"""GPU parity of triangular constant-DD elements (Sec. 3.1, the paper's element) against
the CPU FP64 oracle, through the C-ABI.

* Influence blocks (the closed-form edge sums of the device) equal the oracle's (edge
  integrals by adaptive quadrature) to 1e-11 of each block's largest entry on every pair
  of a triangulated disk -- self terms, neighbours sharing an edge or a vertex -- and of
  two crossing triangulated planes; a receiver on a source edge is reported.
* The H-matrix of a triangle mesh (tree on vertex boxes, ACA, the same product kernels)
  matches the dense oracle product to eps + 1e-6, alone and mixed with rectangles, and
  on 300 sampled rows of a 40,000-triangle fault.
* GMRES on the triangulated penny crack gives the dense LU solution and Sneddon's
  opening to the oracle's discrete error; ILU + BiCGSTAB and point Jacobi + FGMRES on
  its tangent give the LU solution; a batch of a triangle and a rectangle fault gives
  each fault's dense product.
"""
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


def crossing_planes():
    """A triangulated disk z = 0 crossed by a triangulated disk x = 0.013 (jitters differ)."""
    return synth.Elements.concat([synth.tri_disk_mesh(10, seed=1),
                                  synth.tri_disk_mesh(8, radius=0.7, normal=(1, 0, 0), origin=(0.013, 0.0, 0.0),
                                                      seed=2, plane_id=1)])


def gpu_blocks(dev, el, ri, sj):
    import torch
    r = torch.as_tensor(ri, dtype=torch.int64, device=dev)
    s = torch.as_tensor(sj, dtype=torch.int64, device=dev)
    out = torch.empty(ri.size * 9, dtype=torch.float64, device=dev)
    hmat.influence_blocks(el, E, NU, r, s, out)
    return out.cpu().numpy().reshape(-1, 3, 3)


@pytest.mark.parametrize("which", ["disk", "crossing"])
def test_influence_blocks_match_oracle(dev, which):
    el = synth.tri_disk_mesh(12) if which == "disk" else crossing_planes()
    ii, jj = np.meshgrid(np.arange(el.N), np.arange(el.N), indexing="ij")
    ri, sj = ii.ravel(), jj.ravel()
    g = gpu_blocks(dev, el, ri, sj)
    o = O.influence_blocks(el, E, NU, ri, sj)
    scale = np.abs(o).reshape(-1, 9).max(axis=1)
    err = np.abs(g - o).reshape(-1, 9).max(axis=1) / scale
    assert np.all(np.isfinite(g))
    assert err.max() <= 1e-11, (err.max(), np.argmax(err))
    # the self terms: the largest entries, normal-normal negative (compression under opening)
    self_blk = g[ri == sj]
    assert np.all(self_blk[:, 2, 2] < 0)


def test_receiver_on_a_triangle_edge_is_singular(dev):
    import torch
    V0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    # a small triangle whose centroid is the midpoint of V0's first edge
    m = np.array([0.5, 0.0, 0.0])
    V1 = m + np.array([[-0.05, -0.03, 0.0], [0.05, -0.03, 0.0], [0.0, 0.06, 0.0]])
    el = synth.triangles(np.stack([V0, V1]), (0, 0, 1))
    assert np.allclose(el.c[1], m)
    r = torch.tensor([1, 0], dtype=torch.int64, device=dev)
    s = torch.tensor([0, 1], dtype=torch.int64, device=dev)
    out = torch.empty(18, dtype=torch.float64, device=dev)
    with pytest.raises(hmat.HMError) as ei:
        hmat.influence_blocks(el, E, NU, r, s, out)
    assert ei.value.status == hmat.HM_ESINGULAR_GEOM
    o = out.cpu().numpy()
    assert np.all(np.isnan(o[:9])) and np.all(np.isfinite(o[9:]))


def mixed_mesh():
    return synth.Elements.concat([synth.tri_disk_mesh(24),
                                  synth.plane_grid(10, 8, -0.8, 0.8, -0.6, 0.6, (1, 0, 0), origin=(0.013, 0.0, 0.0),
                                                   plane_id=1)])


@pytest.mark.parametrize("name,mk,leaf,eps", [("tripenny", lambda: synth.tri_disk_mesh(28), 32, 1e-6),
                                              ("mixed", mixed_mesh, 48, 1e-6),
                                              ("crossing", crossing_planes, 16, 1e-5)])
def test_matvec_matches_dense_oracle(dev, name, mk, leaf, eps):
    import torch
    el = mk()
    T = hmat.ClusterTree(el, leaf, 2.0)
    H = hmat.HMatrix(T, el, E, NU, eps, "f32")
    A = O.dense_matrix(el, E, NU)
    X = synth.rhs_normal(3 * el.N, 7, nrhs=2)
    for k in range(2):
        ref = A @ X[k]
        for dt in (torch.float32, torch.float64):
            x = torch.as_tensor(X[k], dtype=dt, device=dev)
            y = torch.empty_like(x)
            H.matvec(x, y)
            H.check()
            e = rel(y.cpu().numpy().astype(np.float64), ref)
            assert e <= eps + 1e-6, (name, dt, e)
    print("%s: N = %d, %d leaves" % (name, el.N, T.info()["n_leaves"]))


def test_triangulated_penny_solve(dev):
    import torch
    el = synth.tri_disk_mesh(16)
    T = hmat.ClusterTree(el, 32, 2.0)
    H = hmat.HMatrix(T, el, E, NU, 1e-8, "both")
    b = np.zeros((el.N, 3))
    b[:, 2] = -1.0
    A = O.dense_matrix(el, E, NU)
    xl = np.linalg.solve(A, b.ravel())
    bt = torch.as_tensor(b.ravel(), device=dev)
    for mode in ("f64", "mixed"):
        x = torch.zeros_like(bt)
        info = H.solve(bt, x, torch.zeros(el.N, dtype=torch.float64, device=dev), precond="blockj", mode=mode)[0]
        assert info["status"] == 0 and info["relres"] <= 1e-8
        xs = x.cpu().numpy()
        assert rel(xs, xl) <= 1e-6, (mode, rel(xs, xl))
    r = np.linalg.norm(el.c, axis=1)
    exact = O.sneddon_opening(r, E, NU)
    err_gpu = rel(xs.reshape(-1, 3)[:, 2], exact)
    err_lu = rel(xl.reshape(-1, 3)[:, 2], exact)
    assert abs(err_gpu - err_lu) <= 1e-6 and err_gpu < 0.15
    print("triangulated penny N = %d: Sneddon error %.4f (oracle LU %.4f)" % (el.N, err_gpu, err_lu))


def test_full_size_triangle_fault_sampled_rows(dev):
    """A 40,000-triangle fault (leaf 64, eps 1e-6) on 300 seeded receiver rows against the
    oracle's dense rows: FP64 vectors to eps + 1e-6, FP32 vectors to 2e-5 (the traction of
    the uniform shear nearly cancels inside the fault, so ||E x|| is far below |E| |x|
    and the FP32 rounding of the sums weighs more; measured 8.7e-6)."""
    import torch
    el = synth.tri_disk_mesh(160)
    assert el.N > 39000
    T = hmat.ClusterTree(el, 64, 2.0)
    eps = 1e-6
    H = hmat.HMatrix(T, el, E, NU, eps, "f32")
    x = synth.rhs_shear_plus_bump(el)
    rows = np.sort(np.random.default_rng(9).choice(el.N, 300, replace=False))
    ref = O.dense_matvec_rows(el, E, NU, x, rows)
    dof = (3 * rows[:, None] + np.arange(3)).ravel()
    for dt, bar in ((torch.float64, eps + 1e-6), (torch.float32, 2e-5)):
        xt = torch.as_tensor(x, dtype=dt, device=dev)
        y = torch.empty_like(xt)
        H.matvec(xt, y)
        H.check()
        e = rel(y.cpu().numpy().astype(np.float64)[dof], ref)
        assert e <= bar, (dt, e)
        print("40k triangles, %s vectors: sampled-row error %.2e" % (dt, e))


@pytest.mark.parametrize("precond,method", [("ilu", "bicgstab"), ("jacobi3", "fgmres")])
def test_triangle_tangent_solves_with_the_papers_preconditioners(dev, precond, method):
    """The ILU of Sec. 3.3.1 with BiCGSTAB and the point Jacobi with FGMRES on the tangent
    of a triangulated penny (k log-uniform): the dense LU solution of the oracle's
    tangent."""
    import torch
    el = synth.tri_disk_mesh(14)
    h = 2.0 / 14
    T = hmat.ClusterTree(el, 32, 2.0)
    H = hmat.HMatrix(T, el, E, NU, 1e-8, "both")
    k = synth.k_loguniform(el.N, 1630, E=E, h=h)
    A = O.tangent_dense(O.dense_matrix(el, E, NU), k)
    b = synth.rhs_normal(3 * el.N, 1631)
    x = torch.zeros(3 * el.N, dtype=torch.float64, device=dev)
    info = H.solve(torch.as_tensor(b, device=dev), x, torch.as_tensor(k, device=dev), precond=precond,
                   method=method, ilu_p=0.01)[0]
    assert info["status"] == 0 and info["relres"] <= 1e-8
    assert rel(x.cpu().numpy(), np.linalg.solve(A, b)) <= 1e-6


def test_batch_of_a_triangle_and_a_rectangle_fault(dev):
    """Independent faults of both shapes in one arena: each part of the batched product
    equals the dense oracle product of its fault."""
    import torch
    els = [synth.tri_disk_mesh(20, seed=3), synth.config_penny(18)]
    trees, parts = [], []
    for el in els:
        T = hmat.ClusterTree(el, 32, 2.0)
        trees.append(T)
        parts.append(hmat.HMatrix(T, el, E, NU, 1e-6, "f32"))
    B = hmat.HMatrix.batch(parts)
    n = [3 * el.N for el in els]
    x = synth.rhs_normal(sum(n), 1632)
    xt = torch.as_tensor(x, dtype=torch.float32, device=dev)
    yt = torch.empty_like(xt)
    B.matvec(xt, yt)
    B.check()
    y = yt.cpu().numpy().astype(np.float64)
    off = 0
    for el, nf in zip(els, n):
        ref = O.dense_matrix(el, E, NU) @ x[off:off + nf]
        assert rel(y[off:off + nf], ref) <= 1e-6 + 1e-6
        off += nf
