"""GPU parity of the FP64 influence-block kernel against the CPU oracle, through the
C-ABI (hm_influence_blocks).  Tolerance: 1e-11 of the largest entry of each block
(both sides are FP64; they differ in operation order and FMA contraction only)."""
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


def gpu_blocks(dev, el, ri, sj, E=E, nu=NU):
    import torch
    r = torch.as_tensor(np.asarray(ri, np.int64), device=dev)
    s = torch.as_tensor(np.asarray(sj, np.int64), device=dev)
    out = torch.empty(9 * r.numel(), dtype=torch.float64, device=dev)
    hmat.influence_blocks(el, E, nu, r, s, out)
    return out.cpu().numpy().reshape(-1, 3, 3)


def compare(g, o, tol=1e-11):
    scale = np.abs(o).reshape(len(o), -1).max(axis=1)[:, None, None]
    err = np.abs(g - o) / scale
    assert err.max() <= tol, err.max()


def test_all_pairs_penny(dev):
    el = synth.config_penny(20)
    ii, jj = np.meshgrid(np.arange(el.N), np.arange(el.N), indexing="ij")
    ri, sj = ii.ravel(), jj.ravel()
    compare(gpu_blocks(dev, el, ri, sj), O.influence_blocks(el, E, NU, ri, sj))


def test_random_pairs_three_planes(dev):
    el = synth.config_three_planes(30)
    rng = np.random.default_rng(1)
    ri = rng.integers(0, el.N, 200000)
    sj = rng.integers(0, el.N, 200000)
    compare(gpu_blocks(dev, el, ri, sj), O.influence_blocks(el, E, NU, ri, sj))


def test_crack_fault_intersection_and_poisson(dev):
    el = synth.config_crack_fault(h=0.1)
    rng = np.random.default_rng(2)
    ri = rng.integers(0, el.N, 100000)
    sj = rng.integers(0, el.N, 100000)
    for nu in (0.2, 0.3):
        compare(gpu_blocks(dev, el, ri, sj, 2.0, nu), O.influence_blocks(el, 2.0, nu, ri, sj))


def test_far_pairs_keep_fp64_accuracy(dev):
    el = synth.config_fault(256)
    rng = np.random.default_rng(3)
    ri = rng.integers(0, el.N, 20000)
    sj = rng.integers(0, el.N, 20000)
    compare(gpu_blocks(dev, el, ri, sj), O.influence_blocks(el, E, NU, ri, sj), tol=1e-9)


def test_receiver_on_an_edge_is_an_error(dev):
    el = synth.config_three_planes(8, shift_third=False)
    import torch
    # find a singular pair with the oracle
    N = el.N
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ob = O.influence_blocks(el, E, NU, ii.ravel(), jj.ravel())
    bad = np.where(np.isnan(ob).any(axis=(1, 2)))[0]
    assert bad.size > 0
    r = torch.as_tensor(ii.ravel()[bad[:4]], device=dev)
    s = torch.as_tensor(jj.ravel()[bad[:4]], device=dev)
    out = torch.empty(9 * r.numel(), dtype=torch.float64, device=dev)
    with pytest.raises(hmat.HMError) as ei:
        hmat.influence_blocks(el, E, NU, r, s, out)
    assert ei.value.status == hmat.HM_ESINGULAR_GEOM
    assert torch.isnan(out).all()
