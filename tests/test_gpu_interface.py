"""GPU parity of the interface constitutive update and its consistent tangent
(hm_interface_update; Sec. 2.2, Sec. 3.1.1, eq. jac_mech) against the oracle
(oracle/interface.py), through the C-ABI.

* Every point of 3,001 seeded states (a ragged count) for each material set: the mode
  bit for bit, T'^(n+1), delta^p, (chi_s, chi_t, w_dil) to 1e-12 of the traction and DD
  scales, C^ep to 1e-9 of the largest stiffness (both sides are exact derivatives: dual
  numbers against complex steps).
* 2,000,000 points (the element count of three 800x800 planes) on the launch the
  library uses for every size: the invariants of the law at every point (the active
  yield function vanishes after a return, the elastic law holds on the elastic part of
  the increment, the internal variables bound the magnitudes), and 200 sampled points
  against the oracle.
* Edge cases: no points; in-place update (outputs on the inputs); no tangent and no
  modes requested; the per-mode counts.
"""
import numpy as np
import pytest

from oracle import interface as I
from paper_2605_14397_gb300 import hmat, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def to_dev(dev, *arrs):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in arrs]


@pytest.mark.parametrize("name", list(synth.INTERFACE_PARAMS))
def test_every_point_matches_the_oracle(dev, name):
    kw = synth.INTERFACE_PARAMS[name]
    P = I.Params(**kw)
    n = 3001
    T, dp, chi, dd = synth.interface_states(n, 41)
    T1, dp1, chi1, cep, mode, cnt = hmat.interface_update(kw, *to_dev(dev, T, dp, chi, dd), counts=True)
    T1, dp1, chi1, cep, mode = (x.cpu().numpy() for x in (T1, dp1, chi1, cep, mode))
    rT, rdp, rchi, rmode, rcep = I.step_all(P, T, dp, chi, dd)
    assert np.array_equal(mode, rmode), np.flatnonzero(mode != rmode)[:10]
    assert np.array_equal(cnt[:5], np.bincount(rmode, minlength=5)) and cnt[5] == 0
    assert np.abs(T1 - rT).max() <= 1e-12 * max(1.0, np.abs(rT).max())
    assert np.abs(dp1 - rdp).max() <= 1e-12 * max(0.1, np.abs(rdp).max())
    assert np.abs(chi1 - rchi).max() <= 1e-12 * max(0.1, np.abs(rchi).max())
    scale = max(kw["Ks"], kw["Kn"])
    err = np.abs(cep - rcep).max(axis=(1, 2))
    assert err.max() <= 1e-9 * scale, (err.argmax(), rmode[err.argmax()], err.max())


def test_invariants_at_two_million_points(dev):
    import torch
    kw = synth.INTERFACE_PARAMS["softening"]
    P = I.Params(**kw)
    n = 2_000_000
    T, dp, chi, dd = synth.interface_states(n, 43)
    Td, dpd, chid, ddd = to_dev(dev, T, dp, chi, dd)
    T1, dp1, chi1, cep, mode, cnt = hmat.interface_update(kw, Td, dpd, chid, ddd, counts=False)
    cnt = np.bincount(mode.cpu().numpy() & 255, minlength=5)
    bad = np.flatnonzero(mode.cpu().numpy() >= 256)
    assert bad.size == 0, [(int(e), T[e].tolist(), dp[e].tolist(), chi[e].tolist(), dd[e].tolist())
                           for e in bad[:3]]
    assert cnt.sum() == n and (cnt > 0).sum() >= 4
    K = torch.tensor([kw["Ks"], kw["Ks"], kw["Kn"]], dtype=torch.float64, device=dev)
    m = mode.long()
    notopen = m != I.OPEN
    law = (T1 - (Td + K * (ddd - (dp1 - dpd)))).abs().max(dim=1).values
    assert law[notopen].max().item() <= 1e-12 * max(1.0, T1.abs().max().item())
    assert (T1[m == I.OPEN] == 0).all()

    def soft(scale, x):
        return torch.clamp(1.0 - x / scale, min=0.0)
    f = (kw["fp"] - kw["fr"]) * soft(kw["dc"], chi1[:, 0]) + kw["fr"]
    c = kw["cp"] * soft(kw["wc"], chi1[:, 1])
    st = kw["sigp"] * soft(kw["wc"], chi1[:, 1])
    Fc = torch.hypot(T1[:, 0], T1[:, 1]) + f * T1[:, 2] - c
    Ft = T1[:, 2] - st
    assert Fc[m == I.COULOMB].abs().max().item() <= 1e-12
    assert Fc[m == I.APEX].abs().max().item() <= 1e-12
    assert Ft[m == I.TENSILE].abs().max().item() <= 1e-12
    assert Fc[m == I.ELASTIC].max().item() <= 0 and Ft[m == I.ELASTIC].max().item() <= 0
    assert (chi1[:, 0] >= torch.hypot(dp1[:, 0], dp1[:, 1]) * (1 - 1e-15)).all()
    assert (chi1[:, 1] >= dp1.norm(dim=1) * (1 - 1e-15)).all()
    assert (chi1[:, :2] >= chid[:, :2]).all()
    rng = np.random.default_rng(44)
    idx = np.concatenate([rng.choice(np.flatnonzero(mode.cpu().numpy() == k), 40) for k in (0, 1, 2, 4)] +
                         [rng.choice(n, 40)])
    rT, rdp, rchi, rmode, rcep = I.step_all(P, T[idx], dp[idx], chi[idx], dd[idx])
    assert np.array_equal(mode.cpu().numpy()[idx], rmode)
    assert np.abs(T1.cpu().numpy()[idx] - rT).max() <= 1e-12 * max(1.0, np.abs(rT).max())
    assert np.abs(cep.cpu().numpy()[idx] - rcep).max() <= 1e-9 * kw["Kn"]


def test_edge_cases(dev):
    import torch
    kw = synth.INTERFACE_PARAMS["brittle"]
    z = torch.zeros((0, 3), dtype=torch.float64, device=dev)
    out = hmat.interface_update(kw, z, z, z, z, counts=True)
    assert out[0].shape == (0, 3) and out[5].sum() == 0
    T, dp, chi, dd = synth.interface_states(517, 45)
    Td, dpd, chid, ddd = to_dev(dev, T, dp, chi, dd)
    ref = hmat.interface_update(kw, Td, dpd, chid, ddd)
    bare = hmat.interface_update(kw, Td, dpd, chid, ddd, tangent=False, modes=False)
    assert bare[3] is None and bare[4] is None
    for a, b in zip(ref[:3], bare[:3]):
        assert torch.equal(a, b)
    Tc, dpc, chic = Td.clone(), dpd.clone(), chid.clone()
    hmat.interface_update(kw, Tc, dpc, chic, ddd, T1=Tc, dp1=dpc, chi1=chic)
    assert torch.equal(Tc, ref[0]) and torch.equal(dpc, ref[1]) and torch.equal(chic, ref[2])
