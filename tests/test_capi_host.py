"""C-ABI checks that need no GPU: the library loads, exports every entry point that
include/hmat.h declares, rejects bad arguments with a status code, and its host cluster
tree and block partition are bit-identical to the oracle's."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14397_gb300 import hmat, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(hm_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from __graft_entry__ import build
    build()
    return hmat.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in hmat.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_version_and_error_string(L):
    assert L.hm_version() >= 100
    assert isinstance(hmat.last_error(), str)


def test_bad_arguments_return_status(L):
    h = ctypes.c_void_p()
    assert L.hm_build_cluster_tree(None, 64, 2.0, ctypes.byref(h)) == hmat.HM_EINVAL
    assert "NULL" in hmat.last_error()
    el = synth.config_penny(8)
    ea = hmat._ElemArgs(el)
    assert L.hm_build_cluster_tree(ea.ref, 0, 2.0, ctypes.byref(h)) == hmat.HM_EINVAL
    assert L.hm_build_cluster_tree(ea.ref, 16, -1.0, ctypes.byref(h)) == hmat.HM_EINVAL
    bad = synth.config_penny(8)
    bad.c = bad.c.copy()
    bad.c[3, 1] = np.nan
    eb = hmat._ElemArgs(bad)
    assert L.hm_build_cluster_tree(eb.ref, 16, 2.0, ctypes.byref(h)) == hmat.HM_ENAN
    bad2 = synth.config_penny(8)
    bad2.a = bad2.a.copy()
    bad2.a[0] = 0.0
    assert L.hm_build_cluster_tree(hmat._ElemArgs(bad2).ref, 16, 2.0, ctypes.byref(h)) == hmat.HM_EINVAL
    assert L.hm_matvec(None, None, None, 1, 1, None) == hmat.HM_EINVAL
    assert L.hm_hmat_get_info(None, None) == hmat.HM_EINVAL
    assert L.hm_tree_get_info(None, None) == hmat.HM_EINVAL
    out = ctypes.c_void_p()
    assert L.hm_batch_create(None, 0, None, ctypes.byref(out)) == hmat.HM_EINVAL
    assert L.hm_batch_create(None, 2, None, None) == hmat.HM_EINVAL
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert L.hm_batch_create(nulls, 2, None, ctypes.byref(out)) == hmat.HM_EINVAL and not out.value
    assert L.hm_matvec_graph(None, None, None, 1, 1, None) == hmat.HM_EINVAL
    opt = hmat.hm_assemble_opts(1.0, 0.25, 1e-6, hmat.HM_F32, 0, 0.0)
    buf = ctypes.create_string_buffer(64)
    lv = (ctypes.c_int * 1)(200)
    ev = (ctypes.c_double * 1)(2.0)
    assert L.hm_autotune(ea.ref, ctypes.byref(opt), lv, 1, ev, 1, None, 0, 0, buf, 64, None) == hmat.HM_EINVAL
    assert "leaf" in hmat.last_error()
    assert L.hm_autotune(ea.ref, None, lv, 1, ev, 1, None, 0, 0, buf, 64, None) == hmat.HM_EINVAL
    assert L.hm_autotune(ea.ref, ctypes.byref(opt), lv, 0, ev, 1, None, 0, 0, buf, 64, None) == hmat.HM_EINVAL
    assert L.hm_autotune(ea.ref, ctypes.byref(opt), lv, 1, ev, 1, None, 3, 0, buf, 64, None) == hmat.HM_EINVAL
    assert L.hm_hmat_set_wait(None, 1.0, -1) == hmat.HM_EINVAL
    t = hmat.hm_tile_shape(32768, 128, 4, 16)
    assert L.hm_hmat_set_tile_shape(None, ctypes.byref(t), None) == hmat.HM_EINVAL
    assert L.hm_tune_tile_shape(None, None, 0, 1, buf, 64, None) == hmat.HM_EINVAL


def test_autotune_cache_key_and_hit_without_device(tmp_path, monkeypatch):
    el = synth.config_penny(12)
    k0 = hmat.autotune_key(el, 1.0, 0.25, 1e-6, "f32", (32, 64), (2.0,), "dev")
    assert k0 == hmat.autotune_key(el, 1.0, 0.25, 1e-6, "f32", [32, 64], [2.0], "dev")
    moved = synth.config_penny(12)
    moved.c = moved.c + np.array([0.0, 0.0, 1e-12])
    for other in (hmat.autotune_key(el, 1.0, 0.26, 1e-6, "f32", (32, 64), (2.0,), "dev"),
                  hmat.autotune_key(el, 1.0, 0.25, 1e-6, "bf16", (32, 64), (2.0,), "dev"),
                  hmat.autotune_key(el, 1.0, 0.25, 1e-6, "f32", (64, 32), (2.0,), "dev"),
                  hmat.autotune_key(el, 1.0, 0.25, 1e-6, "f32", (32, 64), (2.0,), "other"),
                  hmat.autotune_key(moved, 1.0, 0.25, 1e-6, "f32", (32, 64), (2.0,), "dev")):
        assert other != k0
    cache = tmp_path / "tune.json"
    stored = {"best": {"leaf": 32, "eta": 2.0, "ms": 1.0}, "candidates": [], "tuned": 2}
    cache.write_text(json.dumps({k0: stored}))

    def no_library():
        raise AssertionError("a cached tuning result must not touch the library")
    monkeypatch.setattr(hmat, "lib", no_library)
    assert hmat.autotune(el, 1.0, 0.25, 1e-6, "f32", (32, 64), (2.0,), cache=str(cache), device="dev") == stored


def _tri_and_rect():
    """A triangulated disk crossed by a plane of rectangles (mixed shapes)."""
    return synth.Elements.concat([synth.tri_disk_mesh(20),
                                  synth.plane_grid(8, 6, -0.8, 0.8, -0.6, 0.6, (1, 0, 0), origin=(0.013, 0.0, 0.0),
                                                   plane_id=1)])


@pytest.mark.parametrize("which,leaf", [("penny", 64), ("penny", 16), ("planes", 32), ("fault", 64),
                                        ("crackfault", 24), ("tripenny", 32), ("mixed", 16)])
def test_tree_and_partition_bit_identical_to_oracle(L, which, leaf):
    el = {"penny": lambda: synth.config_penny(40),
          "planes": lambda: synth.config_three_planes(30),
          "fault": lambda: synth.config_fault(),
          "crackfault": lambda: synth.config_crack_fault(h=0.1),
          "tripenny": lambda: synth.tri_disk_mesh(40),
          "mixed": _tri_and_rect}[which]()
    T = hmat.ClusterTree(el, leaf, 2.0)
    ex = T.export()
    To = O.cluster_tree(el, leaf)
    near, far = O.block_partition(To, 2.0)
    assert np.array_equal(ex["perm"], To.perm)
    assert np.array_equal(ex["begin"], To.begin) and np.array_equal(ex["end"], To.end)
    assert np.array_equal(ex["left"], To.left) and np.array_equal(ex["right"], To.right)
    assert np.array_equal(ex["near"], np.array(near).reshape(-1, 2))
    assert np.array_equal(ex["far"], np.array(far).reshape(-1, 2))
    info = T.info()
    assert info["n_leaves"] == len(To.leaves())


def test_triangle_geometry_checks(L):
    """Triangles are validated on the host: vertices given, finite, non-degenerate, in the
    plane of c and n, around c; the no-allocation entry point takes rectangles only."""
    good = synth.tri_disk_mesh(6)
    hmat.ClusterTree(good, 16, 2.0).close()

    def status(el):
        with pytest.raises(hmat.HMError) as ei:
            hmat.ClusterTree(el, 16, 2.0)
        return ei.value.status

    def variant(fn):
        el = good.subset(np.arange(good.N))
        fn(el)
        return el
    assert status(variant(lambda e: e.tri.__setitem__((3, slice(3, 6)), e.tri[3, 0:3]))) == hmat.HM_EINVAL  # degenerate
    assert status(variant(lambda e: e.tri.__setitem__((4, 2), e.tri[4, 2] + 0.1))) == hmat.HM_EINVAL  # off the plane
    assert status(variant(lambda e: e.c.__setitem__(5, e.tri[5, 0:3] + 2 * (e.tri[5, 0:3] - e.c[5])))) == hmat.HM_EINVAL
    assert status(variant(lambda e: e.tri.__setitem__((6, 1), np.nan))) == hmat.HM_ENAN
    assert status(variant(lambda e: e.shape.__setitem__(7, 5))) == hmat.HM_EINVAL
    # a triangle needs no half sides; a rectangle does
    ok = variant(lambda e: e.a.__setitem__(2, -1.0))
    hmat.ClusterTree(ok, 16, 2.0).close()
    rect = synth.config_penny(6)
    rect.a[0] = 0.0
    assert status(rect) == hmat.HM_EINVAL
    # the struct without vertices
    ea = hmat._ElemArgs(good)
    ea.s.tri = None
    h = ctypes.c_void_p()
    assert L.hm_build_cluster_tree(ea.ref, 16, 2.0, ctypes.byref(h)) == hmat.HM_EINVAL
    # triangles to the no-allocation entry point: refused before any device work
    ea = hmat._ElemArgs(good)
    dummy = ctypes.c_void_p(16)
    assert L.hm_influence_blocks_noalloc(ea.ref, 1.0, 0.25, 0, dummy, dummy, dummy, None) == hmat.HM_EINVAL


def test_learned_model_host_side(tmp_path):
    th = synth.lp_initial_weights(16, seed=3)
    assert hmat.lib().hm_lp_param_count(16) == th.size
    assert hmat.lib().hm_lp_param_count(8) == -1
    with pytest.raises(hmat.HMError) as ei:
        hmat.LearnedCorrection(th, hidden=8)
    assert ei.value.status == hmat.HM_EINVAL
    bad = th.copy()
    bad[5] = np.nan
    with pytest.raises(hmat.HMError) as ei:
        hmat.LearnedCorrection(bad, hidden=16)
    assert ei.value.status == hmat.HM_ENAN
    m = hmat.LearnedCorrection(th, hidden=16)
    assert np.array_equal(m.params(), th.astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(0)
    m.add_samples(rng.normal(size=(5, 8)), rng.uniform(size=(5, 9)))
    m.add_samples(rng.normal(size=(3, 8)), rng.uniform(size=(3, 9)))
    i = m.info()
    assert (i["hidden"], i["n_samples"], i["n_groups"], i["fallback"], i["steps"]) == (16, 8, 2, 0, 0)
    m.set_fallback(True)
    path = tmp_path / "model.hmlp"
    m.save(path)
    r = hmat.LearnedCorrection.load(path)
    assert r.info()["fallback"] == 1 and r.info()["hidden"] == 16
    assert np.array_equal(r.params(), m.params())
    m.clear_samples()
    assert m.info()["n_samples"] == 0
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a model file at all")
    with pytest.raises(hmat.HMError) as ei:
        hmat.LearnedCorrection.load(junk)
    assert ei.value.status == hmat.HM_EINVAL
    # truncated file
    data = path.read_bytes()
    (tmp_path / "short.hmlp").write_bytes(data[:-4])
    with pytest.raises(hmat.HMError):
        hmat.LearnedCorrection.load(tmp_path / "short.hmlp")
    L = hmat.lib()
    assert L.hm_lp_train(None, 1, 1e-3, None, None) == hmat.HM_EINVAL
    assert L.hm_lp_add_samples(m.handle, None, None, 0) == hmat.HM_EINVAL


def test_interface_update_argument_checks(L):
    """Parameter validation happens before any device work; no points is a no-op."""
    good = dict(Ks=10.0, Kn=20.0, fp=0.6, fr=0.3, psip=0.1, dc=0.2, cp=0.1, sigp=0.5, wc=0.4, alphaR=0.5)

    def call(n=0, **kw):
        p = dict(good)
        p.update(kw)
        prm = hmat.hm_interface_params(*[p[k] for k, _ in hmat.hm_interface_params._fields_])
        null = ctypes.c_void_p(None)
        return L.hm_interface_update(ctypes.byref(prm), n, null, null, null, null, null, null, null, null, null,
                                     None, null)
    assert call() == hmat.HM_OK
    for bad in (dict(Ks=0.0), dict(Kn=-1.0), dict(dc=0.0), dict(fp=-0.1), dict(wc=float("nan")),
                dict(sigp=float("inf"))):
        assert call(**bad) == hmat.HM_EINVAL, bad
    assert call(n=-1) == hmat.HM_EINVAL
    assert call(n=5) == hmat.HM_EINVAL and "NULL" in hmat.last_error()
    assert L.hm_interface_update(None, 0, *([ctypes.c_void_p(None)] * 9), None, None) == hmat.HM_EINVAL


def test_flow_create_argument_checks(L):
    """Mesh validation happens on the host before any device work."""
    conn = np.array([[0, 1, 2, 3], [1, 4, 5, 2]], dtype=np.int32)
    a = np.full(2, 0.5)
    b = np.full(2, 0.5)
    h = ctypes.c_void_p()
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    bad = conn.copy()
    bad[1, 2] = 6
    assert L.hm_flow_create(2, vp(bad), 6, vp(a), vp(b), ctypes.byref(h)) == hmat.HM_EINVAL
    bad = conn.copy()
    bad[0, 3] = 0
    assert L.hm_flow_create(2, vp(bad), 6, vp(a), vp(b), ctypes.byref(h)) == hmat.HM_EINVAL
    assert "repeats" in hmat.last_error()
    assert L.hm_flow_create(2, vp(conn), 6, vp(a), vp(-b), ctypes.byref(h)) == hmat.HM_EINVAL
    assert L.hm_flow_create(0, vp(conn), 6, vp(a), vp(b), ctypes.byref(h)) == hmat.HM_EINVAL
    assert L.hm_flow_create(2, None, 6, vp(a), vp(b), ctypes.byref(h)) == hmat.HM_EINVAL
    # a rectangle and a triangle sharing two nodes (hm_flow_create_mesh)
    shape = np.array([0, 1], dtype=np.int32)
    cm = np.array([[0, 1, 2, 3], [1, 4, 2, -1]], dtype=np.int32)
    tri = np.zeros((2, 9))
    tri[1] = [1.0, 0.0, 0.0, 2.0, 0.5, 0.0, 1.0, 1.0, 0.0]

    def mesh(shape_, conn_, tri_):
        return L.hm_flow_create_mesh(2, vp(shape_), vp(conn_), 5, vp(a), vp(b),
                                     vp(tri_) if tri_ is not None else None, ctypes.byref(h))
    bad = cm.copy()
    bad[1, 3] = 0
    assert mesh(shape, bad, tri) == hmat.HM_EINVAL and "fourth" in hmat.last_error()
    flat = tri.copy()
    flat[1, 6:9] = [1.5, 0.25, 0.0]  # collinear with the first two vertices
    assert mesh(shape, cm, flat) == hmat.HM_EINVAL and "degenerate" in hmat.last_error()
    nan = tri.copy()
    nan[1, 4] = np.nan
    assert mesh(shape, cm, nan) == hmat.HM_ENAN
    assert mesh(shape, cm, None) == hmat.HM_EINVAL
    assert mesh(np.array([0, 7], dtype=np.int32), cm, tri) == hmat.HM_EINVAL
    bad = cm.copy()
    bad[1, 2] = 1
    assert mesh(shape, bad, tri) == hmat.HM_EINVAL and "repeats" in hmat.last_error()
