"""GPU parity of the BiCGSTAB tangent solve (HM_METHOD_BICGSTAB; the Krylov method of the
paper's A11 solves, Sec. 3.3.1) against the oracle, through the C-ABI.

* With each preconditioner (the paper's point Jacobi, leaf block-Jacobi, ILU of Sec.
  3.3.1) the solve reaches 1e-8 on the recomputed residual, matches the dense LU solution
  and takes about the iterations of the oracle's BiCGSTAB with the same preconditioner
  (within a quarter or 3: the device preconditioners apply in FP32, BiCGSTAB's
  convergence is irregular).
* Mixed BF16 + FP64 refinement with BiCGSTAB corrections, several right-hand sides and a
  block-diagonal C^ep give the LU solutions as well.
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


@pytest.fixture(scope="module")
def cases(dev):
    out = {}
    for name, (mk, leaf, h) in CASES.items():
        el = mk()
        T = hmat.ClusterTree(el, leaf, 2.0)
        H = hmat.HMatrix(T, el, E, NU, 1e-8, "both")
        k = np.exp(np.random.default_rng(61).uniform(math.log(1e-3), math.log(1e2), size=el.N)) * (E / h)
        out[name] = (el, O.cluster_tree(el, leaf), H, O.dense_matrix(el, E, NU), h, k)
    return out


def oracle_precond(kind, A, At, To, k):
    if kind == "jacobi3":
        inv = O.point_jacobi_inverses(At)
        return lambda r: O.apply_block_jacobi(inv, r)
    if kind == "blockj":
        inv = O.block_jacobi_inverses(At, To)
        return lambda r: O.apply_block_jacobi(inv, r)
    return IL.ilu_preconditioner(A, To, k, 0.01, ordering="colour")[0]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precond", ["jacobi3", "blockj", "ilu"])
def test_bicgstab_matches_lu_and_the_oracle(dev, cases, name, precond):
    import torch
    el, To, H, A, h, k = cases[name]
    At = O.tangent_dense(A, k)
    b = synth.rhs_normal(3 * el.N, 62)
    bt = torch.as_tensor(b, device=dev)
    x = torch.zeros_like(bt)
    info = H.solve(bt, x, torch.as_tensor(k, device=dev), precond=precond, ilu_p=0.01, method="bicgstab",
                   maxit=2000)[0]
    assert info["status"] == 0 and info["relres"] <= 1e-8
    xl = np.linalg.solve(At, b)
    assert np.linalg.norm(x.cpu().numpy() - xl) <= 1e-6 * np.linalg.norm(xl)
    _, its_o, ok = O.bicgstab(lambda v: At @ v, b, oracle_precond(precond, A, At, To, k), tol=1e-8)
    assert ok and abs(info["iters"] - its_o) <= max(3, its_o // 4), (info["iters"], its_o)
    print("%s %s: BiCGSTAB %d iterations (oracle %d)" % (name, precond, info["iters"], its_o))


def test_bicgstab_mixed_several_rhs_and_cep(dev, cases):
    import torch
    el, To, H, A, h, k = cases["penny24"]
    P = IF.Params(**synth.INTERFACE_PARAMS["softening"])
    T, dp, chi, dd = synth.interface_states(el.N, 63)
    cep = IF.step_all(P, T, dp, chi, dd)[4] * (E / h / 20.0)
    At = O.tangent_dense(A, k, 0.0, cep=cep)
    B = synth.rhs_normal(3 * el.N, 64, nrhs=3)
    Bt = torch.as_tensor(B, device=dev).contiguous()
    kt = torch.as_tensor(k, device=dev)
    ct = torch.as_tensor(cep, device=dev).contiguous()
    for mode in ("f64", "mixed"):
        X = torch.zeros_like(Bt)
        infos = H.solve(Bt, X, kt, precond="blockj", mode=mode, method="bicgstab", cep=ct)
        assert all(i["status"] == 0 and i["relres"] <= 1e-8 for i in infos)
        for q in range(3):
            xl = np.linalg.solve(At, B[q])
            assert np.linalg.norm(X[q].cpu().numpy() - xl) <= 1e-6 * np.linalg.norm(xl)


@pytest.mark.parametrize("precond", ["jacobi3", "blockj", "ilu"])
def test_reused_preconditioner_gives_the_same_solution(dev, cases, precond):
    """reuse_precond keeps the preconditioner of the previous call with the same tangent
    inputs: the solution is bit for bit that of a call that builds it."""
    import torch
    el, To, H, A, h, k = cases["penny24"]
    kt = torch.as_tensor(k, device=dev)
    b = torch.as_tensor(synth.rhs_normal(3 * el.N, 65), device=dev)
    x0 = torch.zeros_like(b)
    H.solve(b, x0, kt, precond=precond, ilu_p=0.01)
    x1 = torch.zeros_like(b)
    H.solve(b, x1, kt, precond=precond, ilu_p=0.01, reuse_precond=True)
    assert torch.equal(x0, x1)
    # a different stiffness array is not reused
    k2 = kt * 1.5
    x2 = torch.zeros_like(b)
    x3 = torch.zeros_like(b)
    H.solve(b, x2, k2, precond=precond, ilu_p=0.01, reuse_precond=True)
    H.solve(b, x3, k2, precond=precond, ilu_p=0.01)
    assert torch.equal(x2, x3)
