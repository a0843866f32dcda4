"""The allocation-free influence-block entry point, through the C-ABI.

hm_influence_blocks_noalloc serves callers that may not call cudaMalloc where they
evaluate coefficients (a pooled allocator owning all device memory, a latency-critical
path, a fixed memory budget): it keeps the geometry in a fixed scratch array in the
library's device globals instead of a fresh allocation.  Its blocks must equal those of
hm_influence_blocks (same tolerance as the other kernel tests: 1e-11 of each block's
largest entry) on two calls in a row with different meshes, so the shared scratch left
behind by one call does not leak into the next, and the CPU oracle's blocks on a sample
of the pairs of both calls.  This file is collected last."""
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


def both(dev, el, ri, sj, E=E, nu=NU):
    import torch
    r = torch.as_tensor(np.asarray(ri, np.int64), device=dev)
    s = torch.as_tensor(np.asarray(sj, np.int64), device=dev)
    a = torch.full((9 * r.numel(),), -1.0, dtype=torch.float64, device=dev)
    b = torch.full((9 * r.numel(),), -2.0, dtype=torch.float64, device=dev)
    hmat.influence_blocks(el, E, nu, r, s, a)
    hmat.influence_blocks_noalloc(el, E, nu, r, s, b)
    return a.cpu().numpy().reshape(-1, 3, 3), b.cpu().numpy().reshape(-1, 3, 3)


def close(a, b, tol=1e-11):
    scale = np.abs(a).reshape(len(a), -1).max(axis=1)[:, None, None]
    return (np.abs(a - b) / scale).max() <= tol


def test_matches_allocating_entry_point_on_two_calls_in_a_row(dev):
    # call 1: a crack crossing a fault, all pairs of a subset
    el1 = synth.config_crack_fault(h=0.1)
    rng = np.random.default_rng(21)
    ri1 = rng.integers(0, el1.N, 50000)
    sj1 = rng.integers(0, el1.N, 50000)
    a1, b1 = both(dev, el1, ri1, sj1)
    assert close(a1, b1)
    assert close(O.influence_blocks(el1, E, NU, ri1[:3000], sj1[:3000]), b1[:3000])
    # call 2: a different, larger mesh and other material constants
    el2 = synth.config_three_planes(40)
    ri2 = rng.integers(0, el2.N, 80000)
    sj2 = rng.integers(0, el2.N, 80000)
    a2, b2 = both(dev, el2, ri2, sj2, 2.0, 0.3)
    assert close(a2, b2)
    assert close(O.influence_blocks(el2, 2.0, 0.3, ri2[:3000], sj2[:3000]), b2[:3000])


def test_error_word_is_cleared_between_calls(dev):
    import torch
    bad = synth.config_three_planes(8, shift_third=False)
    ii, jj = np.meshgrid(np.arange(bad.N), np.arange(bad.N), indexing="ij")
    r = torch.as_tensor(ii.ravel(), device=dev)
    s = torch.as_tensor(jj.ravel(), device=dev)
    out = torch.empty(9 * r.numel(), dtype=torch.float64, device=dev)
    with pytest.raises(hmat.HMError) as ei:
        hmat.influence_blocks_noalloc(bad, E, NU, r, s, out)
    assert ei.value.status == hmat.HM_ESINGULAR_GEOM
    good = synth.config_penny(12)
    ri = np.arange(good.N).repeat(good.N)
    sj = np.tile(np.arange(good.N), good.N)
    a, b = both(dev, good, ri, sj)
    assert close(a, b)


def test_rejects_meshes_beyond_the_scratch_limit(dev):
    import torch
    big = synth.config_fault(300)  # about 70,700 elements > 65,536
    assert big.N > 65536
    r = torch.zeros(4, dtype=torch.int64, device=dev)
    out = torch.empty(36, dtype=torch.float64, device=dev)
    with pytest.raises(hmat.HMError) as ei:
        hmat.influence_blocks_noalloc(big, E, NU, r, r, out)
    assert ei.value.status == hmat.HM_EINVAL
    assert "65536" in str(ei.value)
