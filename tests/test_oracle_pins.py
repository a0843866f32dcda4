"""Pins of the CPU oracle against facts it does not compute itself (CPU only).

Each test names the fact it checks.  A plausible mistake in the oracle's kernel (a
dropped term, a sign, a transposed frame, a wrong corner sign) breaks at least one:
  * closed-form self terms of a square element,
  * the coplanar corner formulas of the planar crack (finite-part integrals),
  * brute-force adaptive quadrature of Kelvin's point source (non-coplanar pairs),
  * point-source far-field asymptotics with O((h/r)^2) error,
  * symmetry and translation invariance on uniform planar grids, rotation invariance,
  * continuity of the stress as a parallel receiver plane approaches the source,
  * Sneddon's and Segedin's penny-crack solutions with the error falling under refinement,
    at the discrete values of the survey's independent coplanar computation,
  * the matrix-free row product against the stored dense matrix and against the
    3x3 blocks contracted by numpy (the checker of every full-size product test).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import synth
from tests import pointsource as P

E, NU = 1.0, 0.25
I = np.eye(3)
FR = (I[0], I[1], I[2])


def rand_frame(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return (q[:, 0].copy(), q[:, 1].copy(), q[:, 2].copy())


@pytest.mark.parametrize("h", [0.05, 0.1, 1.0])
@pytest.mark.parametrize("nu", [0.0, 0.25, 0.3])
def test_self_term_square_closed_form(h, nu):
    mu = O.shear_modulus(E, nu)
    st, B = O.influence_point([0, 0, 0], FR, [0, 0, 0], FR, h / 2, h / 2, E, nu)
    assert st == 0
    enn = -2.0 * math.sqrt(2.0) * mu / (math.pi * (1.0 - nu) * h)
    ess = -math.sqrt(2.0) * mu * (2.0 - nu) / (math.pi * (1.0 - nu) * h)
    np.testing.assert_allclose(np.diag(B), [ess, ess, enn], rtol=1e-13)
    off = B - np.diag(np.diag(B))
    assert np.abs(off).max() <= 1e-14 * abs(enn)


def test_self_term_values_for_unit_modulus():
    # h E_nn and h E_ss for E = 1, nu = 0.25 (values of the closed forms to 7 digits)
    st, B = O.influence_point([0, 0, 0], FR, [0, 0, 0], FR, 0.5, 0.5, 1.0, 0.25)
    assert abs(B[2, 2] - (-0.4801687)) < 1e-7
    assert abs(B[0, 0] - (-0.4201476)) < 1e-7


def test_coplanar_corner_formulas():
    rng = np.random.default_rng(11)
    for _ in range(200):
        a, b = rng.uniform(0.02, 0.2, size=2)
        x1, x2 = rng.uniform(-0.8, 0.8, size=2)
        if min(abs(abs(x1) - a), abs(abs(x2) - b)) < 1e-3:
            continue
        st, B = O.influence_point([x1, x2, 0.0], FR, [0, 0, 0], FR, a, b, E, NU)
        C = P.coplanar_closed_form(x1, x2, a, b, E, NU)
        assert st == 0
        assert np.abs(B - C).max() <= 1e-11 * np.abs(C).max()
        # normal and shear are exactly uncoupled in the plane
        assert B[2, 0] == 0.0 and B[2, 1] == 0.0 and B[0, 2] == 0.0 and B[1, 2] == 0.0


def test_brute_force_quadrature_non_coplanar():
    rng = np.random.default_rng(12)
    worst = 0.0
    for _ in range(12):
        rf = rand_frame(rng)
        sf = rand_frame(rng)
        cs = rng.normal(size=3) * 0.1
        a, b = rng.uniform(0.03, 0.1, size=2)
        # receivers from a quarter element to a few elements away, off the source plane
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xr = cs + d * rng.uniform(0.3, 4.0) * max(a, b)
        st, B = O.influence_point(xr, rf, cs, sf, a, b, E, NU)
        Bb = P.brute_block(xr, rf, cs, sf, a, b, E, NU)
        assert st == 0
        worst = max(worst, np.abs(B - Bb).max() / np.abs(Bb).max())
    assert worst < 1e-10


def test_brute_force_intersection_neighbourhood():
    # receivers of one plane at h/2 from a perpendicular plane (fracture intersections)
    h = 0.05
    crack = synth.plane_grid(6, 2, -3 * h, 3 * h, -h, h, (0, 1, 0), plane_id=0)
    fault = synth.plane_grid(6, 6, -3 * h, 3 * h, -3 * h, 3 * h, (1, 0, 0), plane_id=1)
    el = synth.Elements.concat([crack, fault])
    rng = np.random.default_rng(13)
    pairs = [(i, j) for i in range(crack.N) for j in range(crack.N, el.N)]
    pairs += [(j, i) for i in range(crack.N) for j in range(crack.N, el.N)]
    sel = rng.choice(len(pairs), size=16, replace=False)
    ri = np.array([pairs[k][0] for k in sel])
    sj = np.array([pairs[k][1] for k in sel])
    B = O.influence_blocks(el, E, NU, ri, sj)
    for p in range(len(sel)):
        i, j = ri[p], sj[p]
        Bb = P.brute_block(el.c[i], (el.s1[i], el.s2[i], el.n[i]), el.c[j],
                           (el.s1[j], el.s2[j], el.n[j]), el.a[j], el.b[j], E, NU)
        assert np.abs(B[p] - Bb).max() <= 1e-9 * np.abs(Bb).max()


def test_far_field_point_source_asymptotics():
    rng = np.random.default_rng(14)
    rf = rand_frame(rng)
    sf = rand_frame(rng)
    h = 0.1
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    errs = []
    for ratio in (10, 20, 40, 80):
        xr = d * ratio * h
        st, B = O.influence_point(xr, rf, [0, 0, 0], sf, h / 2, h / 2, E, NU)
        Pb = P.point_block(xr, rf, [0, 0, 0], sf, h * h, E, NU)
        errs.append(np.abs(B - Pb).max() / np.abs(Pb).max())
    errs = np.array(errs)
    # error O((h/r)^2): halves twice for every doubling of the distance
    rates = errs[:-1] / errs[1:]
    assert np.all(rates > 3.3) and np.all(rates < 4.7), (errs, rates)
    assert errs[0] < 0.05


def test_symmetry_and_translation_invariance_uniform_grid():
    el = synth.plane_grid(9, 7, -0.45, 0.45, -0.35, 0.35, (0, 0, 1))
    A = O.dense_matrix(el, E, NU)
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    # a block depends only on the centroid offset
    n1 = 9
    def idx(ix, iy):
        return iy * n1 + ix
    B0 = A[3 * idx(2, 3):3 * idx(2, 3) + 3, 3 * idx(5, 1):3 * idx(5, 1) + 3]
    B1 = A[3 * idx(3, 5):3 * idx(3, 5) + 3, 3 * idx(6, 3):3 * idx(6, 3) + 3]
    np.testing.assert_allclose(B0, B1, rtol=1e-12, atol=1e-14 * np.abs(A).max())


def test_symmetry_tilted_plane():
    el = synth.plane_grid(6, 6, -0.3, 0.3, -0.3, 0.3, (1, 1, 0.5), origin=(0.1, -0.2, 0.3))
    A = O.dense_matrix(el, E, NU)
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()


def test_rotation_invariance():
    rng = np.random.default_rng(15)
    el = synth.Elements.concat([
        synth.plane_grid(4, 4, -0.2, 0.2, -0.2, 0.2, (0, 0, 1), plane_id=0),
        synth.plane_grid(4, 4, -0.2, 0.2, -0.2, 0.2, (1, 0, 0), origin=(0.05, 0.0, 0.025), plane_id=1)])
    A = O.dense_matrix(el, E, NU)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    shift = rng.normal(size=3)
    rot = synth.Elements(c=el.c @ Q.T + shift, s1=el.s1 @ Q.T, s2=el.s2 @ Q.T, n=el.n @ Q.T,
                         a=el.a, b=el.b, plane=el.plane)
    B = O.dense_matrix(rot, E, NU)
    assert np.abs(A - B).max() <= 1e-11 * np.abs(A).max()


def test_continuity_towards_the_plane():
    a, b = 0.1, 0.06
    x1, x2 = 0.03, -0.02  # inside the element
    st, B0 = O.influence_point([x1, x2, 0.0], FR, [0, 0, 0], FR, a, b, E, NU)
    errs = []
    for z in (1e-2, 1e-3, 1e-4, 1e-5):
        for sgn in (1.0, -1.0):
            st, Bz = O.influence_point([x1, x2, sgn * z], FR, [0, 0, 0], FR, a, b, E, NU)
            errs.append(np.abs(Bz - B0).max() / np.abs(B0).max())
    errs = np.array(errs).reshape(4, 2)
    assert np.all(np.diff(errs[:, 0]) < 0) and errs[-1].max() < 1e-3


def test_receiver_on_source_edge_is_reported():
    st, B = O.influence_point([0.1, 0.0, 0.0], FR, [0, 0, 0], FR, 0.1, 0.06, E, NU)
    assert st == -4 and np.all(np.isnan(B))
    st, B = O.influence_point([0.05, -0.06, 0.0], FR, [0, 0, 0], FR, 0.1, 0.06, E, NU)
    assert st == -4
    # just off the edge line, out of plane: finite
    st, B = O.influence_point([0.1, 0.0, 1e-3], FR, [0, 0, 0], FR, 0.1, 0.06, E, NU)
    assert st == 0 and np.all(np.isfinite(B))


def _penny_error(n, shear=False):
    el = synth.config_penny(n)
    A = O.dense_matrix(el, E, NU)
    b = np.zeros((el.N, 3))
    if shear:
        b[:, 0] = -1.0
    else:
        b[:, 2] = -1.0
    x = np.linalg.solve(A, b.ravel()).reshape(-1, 3)
    r = np.linalg.norm(el.c, axis=1)
    if shear:
        exact = O.segedin_slip(r, E, NU)
        got = x[:, 0]
    else:
        exact = O.sneddon_opening(r, E, NU)
        got = x[:, 2]
    return np.linalg.norm(got - exact) / np.linalg.norm(exact), x


def test_sneddon_penny_crack_error_falls_with_refinement():
    errs = [_penny_error(n)[0] for n in (10, 20, 40)]  # doubling keeps the staircase edge similar
    assert errs[0] > errs[1] > errs[2]
    # n = 40 (N = 1,264) is a deterministic discrete solution: 0.047096, computed
    # independently from the coplanar closed forms alone; n = 20: 0.0791
    assert abs(errs[2] - 0.047096) < 1e-6
    assert abs(errs[1] - 0.0791) < 5e-5
    e40, x = _penny_error(40)
    # the pressurised crack opens and does not slip
    assert np.all(x[:, 2] > 0) and np.abs(x[:, :2]).max() < 1e-12


def test_segedin_penny_crack_shear_error_falls_with_refinement():
    errs = [_penny_error(n, shear=True)[0] for n in (10, 20, 40)]
    assert errs[0] > errs[1] > errs[2]
    # the same independent computation: 0.0794 (n = 20), 0.0472 (n = 40)
    assert abs(errs[1] - 0.0794) < 5e-5
    assert abs(errs[2] - 0.0472) < 5e-5


def _two_plane_mesh():
    # a crack crossing a fault: E is not symmetric across the two planes
    return synth.Elements.concat([
        synth.plane_grid(6, 4, -0.3, 0.3, -0.2, 0.2, (0, 0, 1), plane_id=0),
        synth.plane_grid(5, 5, -0.25, 0.25, -0.25, 0.25, (1, 0, 0), origin=(0.01, 0.0, 0.013), plane_id=1)])


@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("subset", [False, True])
def test_dense_matvec_rows_equals_stored_dense_product(nrhs, subset):
    """dense_matvec_rows (matrix free, the checker of the full-size tests and the CPU
    baseline) against the stored dense matrix and against the 3x3 blocks of every
    (row, source) pair contracted by numpy: a wrong right-hand-side stride, a sum into
    the wrong row or a transposed block fails here."""
    el = _two_plane_mesh()
    rng = np.random.default_rng(7)
    A = O.dense_matrix(el, E, NU)
    assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()  # the test needs a non-symmetric E
    X = rng.normal(size=(nrhs, 3 * el.N))
    rows = rng.permutation(el.N)[: el.N // 3] if subset else np.arange(el.N)
    Y = O.dense_matvec_rows(el, E, NU, X[0] if nrhs == 1 else X, rows)
    Y = np.atleast_2d(Y)
    assert Y.shape == (nrhs, 3 * rows.size)
    dofs = (3 * rows[:, None] + np.arange(3)).ravel()
    ref = (A[dofs] @ X.T).T
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()
    # independently: the blocks of every (row, source) pair, contracted in numpy
    ri = np.repeat(rows, el.N)
    sj = np.tile(np.arange(el.N), rows.size)
    B = O.influence_blocks(el, E, NU, ri, sj).reshape(rows.size, el.N, 3, 3)
    ref2 = np.einsum("rjam,kjm->kra", B, X.reshape(nrhs, el.N, 3)).reshape(nrhs, -1)
    assert np.abs(Y - ref2).max() <= 1e-13 * np.abs(ref2).max()
