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
    opt = hmat.hm_assemble_opts(1.0, 0.25, 1e-6, hmat.HM_F32, 0)
    buf = ctypes.create_string_buffer(64)
    lv = (ctypes.c_int * 1)(200)
    ev = (ctypes.c_double * 1)(2.0)
    assert L.hm_autotune(ea.ref, ctypes.byref(opt), lv, 1, ev, 1, 0, buf, 64, None) == hmat.HM_EINVAL
    assert "leaf" in hmat.last_error()
    assert L.hm_autotune(ea.ref, None, lv, 1, ev, 1, 0, buf, 64, None) == hmat.HM_EINVAL
    assert L.hm_autotune(ea.ref, ctypes.byref(opt), lv, 0, ev, 1, 0, buf, 64, None) == hmat.HM_EINVAL


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


@pytest.mark.parametrize("which,leaf", [("penny", 64), ("penny", 16), ("planes", 32), ("fault", 64),
                                        ("crackfault", 24)])
def test_tree_and_partition_bit_identical_to_oracle(L, which, leaf):
    el = {"penny": lambda: synth.config_penny(40),
          "planes": lambda: synth.config_three_planes(30),
          "fault": lambda: synth.config_fault(),
          "crackfault": lambda: synth.config_crack_fault(h=0.1)}[which]()
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
