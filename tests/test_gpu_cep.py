"""GPU parity of the tangent solve with a block-diagonal consistent tangent C^ep
(eq. jac_mech: A = E - diag(k) - C^ep - shift I; Sec. 3.3.1 for the preconditioners)
against the oracle, through the C-ABI.

The 3x3 blocks are the oracle's consistent tangents of seeded interface states (Sec. 2.2;
elastic, Coulomb, apex returns: non-symmetric blocks with shear-normal coupling).

* Every preconditioner (none, the paper's point Jacobi, leaf block-Jacobi, ILU) reaches
  1e-8 and matches the dense LU solution of the oracle's tangent; so do the mixed
  BF16 + FP64 refinement and several right-hand sides.
* ILU with C^ep: the pattern holds every element's whole 3x3 block, and the factors equal
  the oracle's ILU(0) of the exported matrix (C^ep entered on the blocks) to 1e-12 of each
  row's largest entry.
* Errors: the learned preconditioner refuses C^ep (HM_EINVAL); a NaN in C^ep is HM_ENAN.
"""
import math

import numpy as np
import pytest

from oracle import ilu as IL
from oracle import interface as IF
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


CASES = {"penny24": (lambda: synth.config_penny(24), 32, 2.0 / 24),
         "crackfault": (lambda: synth.config_crack_fault(h=0.1), 64, 0.1)}


def blocks(N, seed, scale):
    P = IF.Params(**synth.INTERFACE_PARAMS["softening"])
    T, dp, chi, dd = synth.interface_states(N, seed)
    return IF.step_all(P, T, dp, chi, dd)[4] * scale


@pytest.fixture(scope="module")
def cases(dev):
    out = {}
    for name, (mk, leaf, h) in CASES.items():
        el = mk()
        T = hmat.ClusterTree(el, leaf, 2.0)
        H = hmat.HMatrix(T, el, E, NU, 1e-8, "both")
        # blocks on the scale of the elastic diagonal (about E / h)
        cep = blocks(el.N, 51, E / h / 20.0)
        k = np.exp(np.random.default_rng(52).uniform(math.log(1e-3), math.log(1e1), size=el.N)) * (E / h)
        out[name] = (el, O.cluster_tree(el, leaf), H, O.dense_matrix(el, E, NU), h, cep, k)
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precond", ["none", "jacobi3", "blockj", "ilu"])
def test_solve_matches_lu(dev, cases, name, precond):
    import torch
    el, To, H, A, h, cep, k = cases[name]
    shift = 0.1
    At = O.tangent_dense(A, k, shift, cep=cep)
    b = synth.rhs_normal(3 * el.N, 53)
    bt = torch.as_tensor(b, device=dev)
    x = torch.zeros_like(bt)
    info = H.solve(bt, x, torch.as_tensor(k, device=dev), shift=shift, precond=precond, ilu_p=0.05,
                   cep=torch.as_tensor(cep, device=dev).contiguous(), maxit=3000)[0]
    assert info["status"] == 0 and info["relres"] <= 1e-8
    xl = np.linalg.solve(At, b)
    assert np.linalg.norm(x.cpu().numpy() - xl) <= 1e-6 * np.linalg.norm(xl)
    # the device residual of the library agrees with the oracle's tangent
    assert np.linalg.norm(b - At @ x.cpu().numpy()) <= 2e-8 * np.linalg.norm(b)
    print("%s %s: %d iterations" % (name, precond, info["iters"]))


def test_mixed_and_several_rhs(dev, cases):
    import torch
    el, To, H, A, h, cep, k = cases["penny24"]
    At = O.tangent_dense(A, k, 0.0, cep=cep)
    B = synth.rhs_normal(3 * el.N, 54, nrhs=3)
    Bt = torch.as_tensor(B, device=dev).contiguous()
    X = torch.zeros_like(Bt)
    ct = torch.as_tensor(cep, device=dev).contiguous()
    infos = H.solve(Bt, X, torch.as_tensor(k, device=dev), precond="blockj", mode="mixed", cep=ct)
    assert all(i["status"] == 0 for i in infos)
    for q in range(3):
        xl = np.linalg.solve(At, B[q])
        assert np.linalg.norm(X[q].cpu().numpy() - xl) <= 1e-6 * np.linalg.norm(xl)


@pytest.mark.parametrize("name", list(CASES))
def test_ilu_with_cep_matches_the_oracle(dev, cases, name):
    import torch
    el, To, H, A, h, cep, k = cases[name]
    shift = 0.2
    ex = H.ilu_export(torch.as_tensor(k, device=dev), shift, p=0.01,
                      cep=torch.as_tensor(cep, device=dev).contiguous())
    order, rp, col, aval, lu = ex["order"], ex["rowptr"], ex["col"], ex["a_val"], ex["lu_val"]
    n = order.size
    perm = np.asarray(To.perm)
    rows = []
    for a in range(n):
        r = {int(col[q]): aval[q] for q in range(rp[a], rp[a + 1])}
        ra = int(order[a])
        qa = ra // 3
        # every entry of the element's block is in the pattern
        blk = [c for c, _ in r.items() if int(order[c]) // 3 == qa]
        assert len(blk) == 3, (a, blk)
        for c in blk:
            r[c] -= cep[perm[qa], ra % 3, int(order[c]) % 3]
        r[a] -= k[perm[qa]] + shift
        rows.append(r)
    L, U = IL.ilu0(rows)
    for a in range(n):
        scale = max(abs(x) for x in rows[a].values())
        for q in range(rp[a], rp[a + 1]):
            c = int(col[q])
            ref = L[a][c] if c < a else U[a][c]
            assert abs(lu[q] - ref) <= 1e-12 * max(scale, abs(ref)), (a, c, lu[q], ref)
    # the same pattern as the oracle's sparse approximation with C^ep (selection from the
    # FP32 store, up to a handful of rounding-boundary entries)
    ref_rows = IL.sparse_tangent(A.astype(np.float32).astype(np.float64), To, k, p=0.01, shift=shift, cep=cep)
    lib = {(int(order[a]), int(order[col[q]])) for a in range(n) for q in range(rp[a], rp[a + 1])}
    ref = {(a, c) for a in range(n) for c in ref_rows[a]}
    assert len(lib ^ ref) <= 2 + 1e-3 * len(ref)


def test_errors(dev, cases):
    import torch
    el, To, H, A, h, cep, k = cases["penny24"]
    b = torch.as_tensor(synth.rhs_normal(3 * el.N, 55), device=dev)
    x = torch.zeros_like(b)
    ct = torch.as_tensor(cep, device=dev).contiguous()
    lp = hmat.LearnedCorrection(synth.lp_initial_weights(hidden=16), hidden=16)
    with pytest.raises(hmat.HMError) as e:
        H.solve(b, x, None, precond="learned", model=lp, cep=ct)
    assert e.value.status == hmat.HM_EINVAL
    bad = ct.clone()
    bad[3, 1, 2] = float("nan")
    with pytest.raises(hmat.HMError) as e:
        H.solve(b, x, None, precond="blockj", cep=bad)
    assert e.value.status == hmat.HM_ENAN
