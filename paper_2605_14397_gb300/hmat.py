"""Thin Python binding of libhmat (include/hmat.h).  Argument marshalling only: every
step of the hot path runs in the CUDA library.  PyTorch supplies device memory and
streams; there is no CPU fallback -- if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmat.so")

HM_OK = 0
HM_EINVAL = -1
HM_ENOMEM = -2
HM_ECUDA = -3
HM_ESINGULAR_GEOM = -4
HM_ENOCONV = -5
HM_EBREAKDOWN = -6
HM_ENAN = -7
HM_ETIMEOUT = -8
HM_F32, HM_F64, HM_BF16, HM_F32_BF16 = 1, 2, 3, 4
HM_PRECOND_NONE, HM_PRECOND_BLOCKJ, HM_PRECOND_LEARNED, HM_PRECOND_JACOBI3, HM_PRECOND_ILU = 0, 1, 2, 3, 4
HM_SOLVE_F64, HM_SOLVE_MIXED, HM_SOLVE_PLAIN32 = 1, 2, 3
HM_METHOD_FGMRES, HM_METHOD_BICGSTAB = 0, 1
HM_LP_SCALE, HM_LP_NEAR = 0, 1

_STATUS_NAMES = {HM_EINVAL: "HM_EINVAL", HM_ENOMEM: "HM_ENOMEM", HM_ECUDA: "HM_ECUDA",
                 HM_ESINGULAR_GEOM: "HM_ESINGULAR_GEOM", HM_ENOCONV: "HM_ENOCONV",
                 HM_EBREAKDOWN: "HM_EBREAKDOWN", HM_ENAN: "HM_ENAN", HM_ETIMEOUT: "HM_ETIMEOUT"}


class HMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (_STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class hm_elements(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64)] + [(n, ctypes.POINTER(ctypes.c_double))
                                           for n in ("c", "s1", "s2", "n", "a", "b")] + [
        ("shape", ctypes.POINTER(ctypes.c_int32)), ("tri", ctypes.POINTER(ctypes.c_double))]


class hm_tree_info(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_near", ctypes.c_int64), ("n_far", ctypes.c_int64), ("leaf_size", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("eta", ctypes.c_double)]


class hm_assemble_opts(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("aca_eps", ctypes.c_double),
                ("storage", ctypes.c_int), ("max_rank", ctypes.c_int), ("trunc_factor", ctypes.c_double)]


class hm_hmat_info(ctypes.Structure):
    _fields_ = [("n_dof", ctypes.c_int64), ("near_entries", ctypes.c_int64), ("far_entries", ctypes.c_int64),
                ("stored_bytes", ctypes.c_int64), ("algorithmic_bytes", ctypes.c_int64),
                ("rank_min", ctypes.c_int32), ("rank_max", ctypes.c_int32), ("rank_mean", ctypes.c_double),
                ("assemble_seconds", ctypes.c_double), ("storage", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("n_far_lowrank", ctypes.c_int64), ("n_far_dense", ctypes.c_int64),
                ("u_entries", ctypes.c_int64), ("v_entries", ctypes.c_int64), ("tb_len", ctypes.c_int64),
                ("p_len", ctypes.c_int64), ("n_far_refined", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("coeff_blocks", ctypes.c_int64)]


class hm_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("precond", ctypes.c_int), ("mode", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("pad_", ctypes.c_int), ("lp", ctypes.c_void_p),
                ("ilu_p", ctypes.c_double), ("cep_dev", ctypes.c_void_p), ("method", ctypes.c_int),
                ("reuse_precond", ctypes.c_int)]


class hm_tile_shape(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_int32), ("chunk_cols", ctypes.c_int32), ("ring", ctypes.c_int32),
                ("warps", ctypes.c_int32)]


DEFAULT_SHAPES = [(32768, 128, 4, 16), (16384, 128, 4, 16), (32768, 64, 4, 16), (16384, 64, 6, 16),
                  (32768, 128, 6, 16), (32768, 128, 4, 8), (16384, 64, 4, 8), (8192, 32, 6, 16)]


def _shape_array(shapes):
    arr = (hm_tile_shape * len(shapes))()
    for q, t in enumerate(shapes):
        arr[q] = hm_tile_shape(*[int(v) for v in t])
    return arr


class hm_lp_info(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("fallback", ctypes.c_int32), ("n_params", ctypes.c_int64),
                ("n_samples", ctypes.c_int64), ("n_groups", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("last_loss", ctypes.c_double), ("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("gamma", ctypes.c_double)]


class hm_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("status", ctypes.c_int), ("pad_", ctypes.c_int),
                ("relres", ctypes.c_double), ("seconds", ctypes.c_double)]


class hm_interface_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("Ks", "Kn", "fp", "fr", "psip", "dc", "cp", "sigp", "wc", "alphaR")]


class hm_flow_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mu", "M", "w0", "dt")]


class hm_coupled_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("inner_precond", ctypes.c_int), ("inner_method", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("schur_tol", ctypes.c_double), ("ilu_p", ctypes.c_double), ("flow_scale", ctypes.c_double)]


class hm_coupled_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("schur_iters", ctypes.c_int),
                ("status", ctypes.c_int), ("relres", ctypes.c_double), ("seconds", ctypes.c_double)]


_LIB = None

# (name, restype, argtypes) of every exported entry point declared in include/hmat.h
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_I = ctypes.c_int
_P64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("hm_last_error", ctypes.c_char_p, []),
    ("hm_version", ctypes.c_int, []),
    ("hm_influence_blocks", _I, [ctypes.POINTER(hm_elements), _D, _D, _I64, _VP, _VP, _VP, _VP]),
    ("hm_influence_blocks_noalloc", _I, [ctypes.POINTER(hm_elements), _D, _D, _I64, _VP, _VP, _VP, _VP]),
    ("hm_build_cluster_tree", _I, [ctypes.POINTER(hm_elements), _I, _D, ctypes.POINTER(_VP)]),
    ("hm_tree_get_info", _I, [_VP, ctypes.POINTER(hm_tree_info)]),
    ("hm_tree_export", _I, [_VP, _P64, _P64, _P64, _P64, _P64, _P64, _P64]),
    ("hm_tree_destroy", None, [_VP]),
    ("hm_assemble_hmat", _I, [_VP, ctypes.POINTER(hm_elements), ctypes.POINTER(hm_assemble_opts), _VP,
                              ctypes.POINTER(_VP)]),
    ("hm_hmat_get_info", _I, [_VP, ctypes.POINTER(hm_hmat_info)]),
    ("hm_hmat_far_factors", _I, [_VP, _I64, ctypes.POINTER(ctypes.c_int32), _VP, _VP]),
    ("hm_hmat_destroy", None, [_VP]),
    ("hm_matvec", _I, [_VP, _VP, _VP, _I, _I, _VP]),
    ("hm_hmat_check", _I, [_VP, _VP]),
    ("hm_hmat_set_wait", _I, [_VP, _D, _I64]),
    ("hm_matvec_host", _I, [_VP, _VP, _VP, _I, _I, _VP]),
    ("hm_matvec_factors", _I, [_VP, _VP, _VP, _I, _I, _I, _VP]),
    ("hm_hmat_timing", _I, [_VP, _I]),
    ("hm_hmat_timing_read", _I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    ("hm_gmres_solve", _I, [_VP, _VP, _D, _VP, _VP, _I, ctypes.POINTER(hm_solve_opts),
                            ctypes.POINTER(hm_solve_info), _VP]),
    ("hm_batch_create", _I, [ctypes.POINTER(_VP), _I, _VP, ctypes.POINTER(_VP)]),
    ("hm_ilu_apply", _I, [_VP, _VP, _VP, _I, _VP]),
    ("hm_ilu_export", _I, [_VP, _VP, _VP, _D, _D, _P64, _P64, ctypes.POINTER(ctypes.c_int32), _VP, _VP, _VP, _VP, _VP,
                           _VP]),
    ("hm_lp_param_count", _I64, [_I]),
    ("hm_lp_create", _I, [_I, _VP, ctypes.POINTER(_VP)]),
    ("hm_lp_add_samples", _I, [_VP, _VP, _VP, _I64]),
    ("hm_lp_add_system", _I, [_VP, _VP, _VP, _VP, _VP, _I, _VP]),
    ("hm_lp_clear_samples", _I, [_VP]),
    ("hm_lp_loss_grad", _I, [_VP, ctypes.POINTER(_D), _VP, _VP]),
    ("hm_lp_train", _I, [_VP, _I, _D, ctypes.POINTER(_D), _VP]),
    ("hm_lp_predict", _I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    ("hm_lp_get_params", _I, [_VP, _VP]),
    ("hm_lp_set_fallback", _I, [_VP, _I]),
    ("hm_lp_get_info", _I, [_VP, ctypes.POINTER(hm_lp_info)]),
    ("hm_lp_set_kind", _I, [_VP, _I, _D]),
    ("hm_precond_apply", _I, [_VP, _VP, _D, ctypes.POINTER(hm_solve_opts), _VP, _VP, _I, _VP]),
    ("hm_lp_save", _I, [_VP, ctypes.c_char_p]),
    ("hm_lp_load", _I, [ctypes.c_char_p, ctypes.POINTER(_VP)]),
    ("hm_lp_destroy", None, [_VP]),
    ("hm_matvec_graph", _I, [_VP, _VP, _VP, _I, _I, _VP]),
    ("hm_autotune", _I, [ctypes.POINTER(hm_elements), ctypes.POINTER(hm_assemble_opts), ctypes.POINTER(_I), _I,
                         ctypes.POINTER(_D), _I, _VP, _I, _I, ctypes.c_char_p, ctypes.c_size_t, _VP]),
    ("hm_hmat_set_tile_shape", _I, [_VP, ctypes.POINTER(hm_tile_shape), _VP]),
    ("hm_hmat_get_tile_shape", _I, [_VP, ctypes.POINTER(hm_tile_shape)]),
    ("hm_tune_tile_shape", _I, [_VP, _VP, _I, _I, ctypes.c_char_p, ctypes.c_size_t, _VP]),
    ("hm_flow_create", _I, [_I64, _VP, _I64, _VP, _VP, ctypes.POINTER(_VP)]),
    ("hm_flow_create_mesh", _I, [_I64, _VP, _VP, _I64, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    ("hm_flow_destroy", None, [_VP]),
    ("hm_flow_assemble", _I, [_VP, ctypes.POINTER(hm_flow_params), _VP, _VP, _VP, _VP]),
    ("hm_flow_export", _I, [_VP, _P64, _VP, _VP, _VP, _VP, _VP]),
    ("hm_coupled_matvec", _I, [_VP, _VP, _VP, _VP, _D, _VP, _VP, _VP]),
    ("hm_coupled_solve", _I, [_VP, _VP, _VP, _VP, _D, _VP, _VP, ctypes.POINTER(hm_coupled_opts),
                              ctypes.POINTER(hm_coupled_info), _VP]),
    ("hm_interface_update", _I, [ctypes.POINTER(hm_interface_params), _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                 _VP, _VP, _P64, _VP]),
    ("hm_ilu_select", _I, [_I64, _VP, _VP, _VP, _D, _VP, ctypes.POINTER(_I64)]),
    ("hm_ilu_assemble", _I, [ctypes.c_int32, _I64, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                             ctypes.POINTER(_I64)]),
    ("hm_ilu0_factor", _I, [ctypes.c_int32, _VP, _VP, _VP]),
    ("hm_ilu_levels", _I, [ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32)]),
    ("hm_ilu_leaf_colours", _I, [ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32, _VP,
                                 ctypes.POINTER(ctypes.c_int32)]),
]


def lib():
    """Load libhmat.so (built by __graft_entry__.build() / paper_2605_14397_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhmat.so is not built (run __graft_entry__.build()); "
                              "there is no CPU fallback for the hot path")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status):
    if status != HM_OK:
        raise HMError(status, lib().hm_last_error().decode())


def last_error() -> str:
    return lib().hm_last_error().decode()


class _ElemArgs:
    """Keeps the contiguous FP64 arrays alive while the struct points at them."""

    def __init__(self, el):
        self.arrs = [np.ascontiguousarray(getattr(el, k), dtype=np.float64) for k in ("c", "s1", "s2", "n", "a", "b")]
        dp = ctypes.POINTER(ctypes.c_double)
        ptrs = [a.ctypes.data_as(dp) for a in self.arrs]
        shape = getattr(el, "shape", None)
        if shape is not None and np.any(np.asarray(shape) != 0):
            self.shape = np.ascontiguousarray(shape, dtype=np.int32)
            self.tri = np.ascontiguousarray(el.tri, dtype=np.float64)
            ptrs += [self.shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.tri.ctypes.data_as(dp)]
        else:
            ptrs += [None, None]
        self.s = hm_elements(el.N, *ptrs)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ entry points

def influence_blocks(el, E, nu, ri, sj, out, stream=None):
    """Fill out (npairs*9 float64, device) with the 3x3 blocks E_{ri[p], sj[p]}."""
    ea = _ElemArgs(el)
    _check(lib().hm_influence_blocks(ea.ref, float(E), float(nu), int(ri.numel()), _dptr(ri), _dptr(sj),
                                     _dptr(out), ctypes.c_void_p(_stream_ptr(stream))))


def influence_blocks_noalloc(el, E, nu, ri, sj, out, stream=None):
    """influence_blocks without device allocation: for callers that may not call
    cudaMalloc (pooled allocators, latency-critical paths, fixed memory budgets).
    Uses the library's fixed 8 MiB device scratch, so el.N <= 65,536; calls that overlap
    on the GPU race on that scratch."""
    ea = _ElemArgs(el)
    _check(lib().hm_influence_blocks_noalloc(ea.ref, float(E), float(nu), int(ri.numel()), _dptr(ri), _dptr(sj),
                                             _dptr(out), ctypes.c_void_p(_stream_ptr(stream))))


class ClusterTree:
    def __init__(self, el, leaf_size=64, eta=2.0):
        ea = _ElemArgs(el)
        h = ctypes.c_void_p()
        _check(lib().hm_build_cluster_tree(ea.ref, int(leaf_size), float(eta), ctypes.byref(h)))
        self.handle = h

    def info(self):
        i = hm_tree_info()
        _check(lib().hm_tree_get_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in hm_tree_info._fields_}

    def export(self):
        i = self.info()
        nn, ne = i["n_nodes"], i["n_elements"]
        perm = np.empty(ne, np.int64)
        begin, end, left, right = (np.empty(nn, np.int64) for _ in range(4))
        near = np.empty((max(i["n_near"], 1), 2), np.int64)
        far = np.empty((max(i["n_far"], 1), 2), np.int64)
        p = lambda a: a.ctypes.data_as(_P64)
        _check(lib().hm_tree_export(self.handle, p(perm), p(begin), p(end), p(left), p(right), p(near), p(far)))
        return dict(perm=perm, begin=begin, end=end, left=left, right=right,
                    near=near[:i["n_near"]], far=far[:i["n_far"]])

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().hm_tree_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HMatrix:
    def __init__(self, tree, el, E=1.0, nu=0.25, aca_eps=1e-6, storage="f32", max_rank=0, stream=None,
                 trunc_factor=0.0):
        st = {"f32": HM_F32, "bf16": HM_BF16, "both": HM_F32_BF16}[storage]
        ea = _ElemArgs(el) if el is not None else None
        opt = hm_assemble_opts(float(E), float(nu), float(aca_eps), st, int(max_rank), float(trunc_factor))
        h = ctypes.c_void_p()
        _check(lib().hm_assemble_hmat(tree.handle, ea.ref if ea else None, ctypes.byref(opt),
                                      ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self.handle = h
        self.E, self.nu, self.eps, self.storage = E, nu, aca_eps, storage
        self.ndof = 3 * el.N if el is not None else None

    @classmethod
    def batch(cls, parts, stream=None):
        """One H-matrix of independent faults (block-diagonal operator): the parts'
        vectors back to back, one work list for the whole batch.  The parts are copied
        and stay usable."""
        parts = list(parts)
        arr = (_VP * len(parts))(*[p.handle.value for p in parts])
        h = ctypes.c_void_p()
        _check(lib().hm_batch_create(arr, len(parts), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle = h
        self.E = self.nu = None
        self.eps = max(p.eps for p in parts)
        self.storage = parts[0].storage
        self.ndof = sum(p.ndof for p in parts)
        return self

    def info(self):
        i = hm_hmat_info()
        _check(lib().hm_hmat_get_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in hm_hmat_info._fields_}

    def far_factors(self, b):
        r = ctypes.c_int32()
        _check(lib().hm_hmat_far_factors(self.handle, int(b), ctypes.byref(r), None, None))
        return r.value

    def far_factor_arrays(self, b, s_n, t_n):
        """(U, V) of far block b, or None if the block is stored dense or was refined."""
        r = self.far_factors(b)
        if r < 0:
            return None
        U = np.empty((r, 3 * s_n))
        V = np.empty((r, 3 * t_n))
        _check(lib().hm_hmat_far_factors(self.handle, int(b), None, U.ctypes.data_as(_VP), V.ctypes.data_as(_VP)))
        return U.T, V.T  # column-major on the C side -> (3|s| x r), (3|t| x r)

    def matvec(self, x, y, stream=None, factors=None):
        """y = E x; x, y torch CUDA tensors of shape (3N,) or (nrhs, 3N), float32 or float64;
        factors "f32" or "bf16" picks a stored factor precision (default: FP32 when stored)."""
        import torch
        dt = {torch.float32: HM_F32, torch.float64: HM_F64}[x.dtype]
        assert y.dtype == x.dtype and x.is_contiguous() and y.is_contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if factors is None:
            _check(lib().hm_matvec(self.handle, _dptr(x), _dptr(y), int(nrhs), dt,
                                   ctypes.c_void_p(_stream_ptr(stream))))
        else:
            fc = {"f32": HM_F32, "bf16": HM_BF16}[factors]
            _check(lib().hm_matvec_factors(self.handle, _dptr(x), _dptr(y), int(nrhs), dt, fc,
                                           ctypes.c_void_p(_stream_ptr(stream))))

    def matvec_graph(self, x, y, stream=None):
        """matvec replayed from a CUDA graph instantiated for these (x, y) on first use."""
        import torch
        dt = {torch.float32: HM_F32, torch.float64: HM_F64}[x.dtype]
        assert y.dtype == x.dtype and x.is_contiguous() and y.is_contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        _check(lib().hm_matvec_graph(self.handle, _dptr(x), _dptr(y), int(nrhs), dt,
                                     ctypes.c_void_p(_stream_ptr(stream))))

    def matvec_host(self, x, y, stream=None):
        """y = E x for host numpy arrays (float32 or float64); synchronous."""
        dt = {np.dtype(np.float32): HM_F32, np.dtype(np.float64): HM_F64}[x.dtype]
        assert y.dtype == x.dtype and x.flags.c_contiguous and y.flags.c_contiguous
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        _check(lib().hm_matvec_host(self.handle, x.ctypes.data_as(_VP), y.ctypes.data_as(_VP), int(nrhs), dt,
                                    ctypes.c_void_p(_stream_ptr(stream))))

    def solve(self, b, x, k=None, shift=0.0, tol=1e-8, restart=50, maxit=2000, precond="blockj", mode="f64",
              inner_tol=1e-2, max_outer=40, stream=None, raise_on_error=True, model=None, ilu_p=0.0, cep=None,
              method="fgmres", reuse_precond=False):
        """Solve (E - diag(k) - C^ep - shift I) x = b on the device (b, x: float64 CUDA tensors
        of shape (3N,) or (nrhs, 3N); k: float64 CUDA tensor (N,) or None; cep: float64 CUDA
        tensor (N, 3, 3) of per-element tangent blocks, user order, or None).  precond "none",
        "jacobi3", "blockj", "ilu" (ilu_p: fraction of the near field, 0 = 0.01) or "learned";
        mode "f64", "mixed" or "plain32"; method "fgmres" or "bicgstab".  Returns the
        per-RHS info dicts; raises HMError unless every RHS converged (raise_on_error)."""
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        assert b.is_contiguous() and x.is_contiguous() and (k is None or k.is_contiguous())
        assert cep is None or (cep.is_contiguous() and cep.numel() == 3 * self.ndof)
        o = hm_solve_opts(float(tol), int(restart), int(maxit),
                          {"none": HM_PRECOND_NONE, "blockj": HM_PRECOND_BLOCKJ, "learned": HM_PRECOND_LEARNED,
                           "jacobi3": HM_PRECOND_JACOBI3, "ilu": HM_PRECOND_ILU}[precond],
                          {"f64": HM_SOLVE_F64, "mixed": HM_SOLVE_MIXED, "plain32": HM_SOLVE_PLAIN32}[mode],
                          float(inner_tol), int(max_outer), 0,
                          model.handle.value if model is not None else None, float(ilu_p),
                          cep.data_ptr() if cep is not None else None,
                          {"fgmres": HM_METHOD_FGMRES, "bicgstab": HM_METHOD_BICGSTAB}[method], int(bool(reuse_precond)))
        info = (hm_solve_info * nrhs)()
        st = lib().hm_gmres_solve(self.handle, _dptr(k) if k is not None else None, float(shift), _dptr(b), _dptr(x),
                                  int(nrhs), ctypes.byref(o), info, ctypes.c_void_p(_stream_ptr(stream)))
        out = [{f: getattr(i, f) for f, _ in hm_solve_info._fields_ if f != "pad_"} for i in info]
        if st != HM_OK and raise_on_error:
            raise HMError(st, lib().hm_last_error().decode())
        return out

    def precond_apply(self, r, z, k=None, shift=0.0, precond="blockj", ilu_p=0.0, cep=None, model=None,
                      reuse_precond=False, stream=None):
        """z = M^-1 r with the preconditioner of solve() for these arguments
        (hm_precond_apply); r, z float64 CUDA tensors (3N,) or (nrhs, 3N)."""
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        assert r.is_contiguous() and z.is_contiguous()
        o = hm_solve_opts(0.0, 0, 0,
                          {"none": HM_PRECOND_NONE, "blockj": HM_PRECOND_BLOCKJ, "learned": HM_PRECOND_LEARNED,
                           "jacobi3": HM_PRECOND_JACOBI3, "ilu": HM_PRECOND_ILU}[precond], HM_SOLVE_F64, 0.0, 0, 0,
                          model.handle.value if model is not None else None, float(ilu_p),
                          cep.data_ptr() if cep is not None else None, 0, int(bool(reuse_precond)))
        _check(lib().hm_precond_apply(self.handle, _dptr(k) if k is not None else None, float(shift), ctypes.byref(o),
                                      _dptr(r), _dptr(z), int(nrhs), ctypes.c_void_p(_stream_ptr(stream))))

    def ilu_export(self, k=None, shift=0.0, p=0.01, factor=True, stream=None, cep=None):
        """The ILU preconditioner for this k, C^ep, shift and p (hm_ilu_export): dict of order
        (factorization position -> cluster DOF position), rowptr, col, a_val and, with
        factor, lu_val, plus n_colours."""
        n, nnz, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        kp = _dptr(k) if k is not None else None
        cp = _dptr(cep) if cep is not None else None
        sp = ctypes.c_void_p(_stream_ptr(stream))
        _check(lib().hm_ilu_export(self.handle, kp, cp, float(shift), float(p), ctypes.byref(n), ctypes.byref(nnz),
                                   ctypes.byref(nc), None, None, None, None, None, sp))
        order = np.empty(n.value, np.int32)
        rowptr = np.empty(n.value + 1, np.int64)
        col = np.empty(nnz.value, np.int32)
        aval = np.empty(nnz.value)
        lu = np.empty(nnz.value) if factor else None
        _check(lib().hm_ilu_export(self.handle, kp, cp, float(shift), float(p), ctypes.byref(n), ctypes.byref(nnz),
                                   ctypes.byref(nc), order.ctypes.data_as(_VP), rowptr.ctypes.data_as(_VP),
                                   col.ctypes.data_as(_VP), aval.ctypes.data_as(_VP),
                                   lu.ctypes.data_as(_VP) if factor else None, sp))
        return dict(order=order, rowptr=rowptr, col=col, a_val=aval, lu_val=lu, n_colours=nc.value)

    def set_tile_shape(self, shape, stream=None):
        """shape: (chunk_bytes, chunk_cols, ring, warps); the product plans are cut again."""
        t = hm_tile_shape(*[int(v) for v in shape])
        _check(lib().hm_hmat_set_tile_shape(self.handle, ctypes.byref(t), ctypes.c_void_p(_stream_ptr(stream))))

    def tile_shape(self):
        t = hm_tile_shape()
        _check(lib().hm_hmat_get_tile_shape(self.handle, ctypes.byref(t)))
        return (t.chunk_bytes, t.chunk_cols, t.ring, t.warps)

    def tune_tile_shape(self, shapes=None, reps=20, stream=None):
        """Time the single-RHS product under each shape and keep the fastest (hm_tune_tile_shape)."""
        import json
        shapes = list(shapes or DEFAULT_SHAPES)
        arr = _shape_array(shapes)
        cap = 1024 + 160 * len(shapes)
        buf = ctypes.create_string_buffer(cap)
        _check(lib().hm_tune_tile_shape(self.handle, arr, len(shapes), int(reps), buf, cap,
                                        ctypes.c_void_p(_stream_ptr(stream))))
        return json.loads(buf.value.decode())

    def ilu_apply(self, r, z, stream=None):
        """z = (L U)^-1 r with the last ILU factorization (float64 CUDA tensors (3N,) or (nrhs, 3N))."""
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        assert r.is_contiguous() and z.is_contiguous()
        _check(lib().hm_ilu_apply(self.handle, _dptr(r), _dptr(z), int(nrhs), ctypes.c_void_p(_stream_ptr(stream))))

    def timing(self, enable):
        _check(lib().hm_hmat_timing(self.handle, 1 if enable else 0))

    def timing_read(self):
        """Milliseconds summed per phase: gather, phase1, reduce, phase2, scatter, count."""
        out = (ctypes.c_double * 6)()
        _check(lib().hm_hmat_timing_read(self.handle, out))
        return dict(gather=out[0], phase1=out[1], reduce=out[2], phase2=out[3], scatter=out[4], count=int(out[5]))

    def set_wait(self, limit_s=2.0, withhold_chunk=-1):
        """Limit of the product's bounded waits; withhold_chunk >= 0 is a test switch that makes
        the row phase's producer stop before that chunk, so that the waits run out."""
        _check(lib().hm_hmat_set_wait(self.handle, float(limit_s), int(withhold_chunk)))

    def check(self, stream=None):
        """Synchronise and raise HMError(HM_ETIMEOUT) if a product kernel gave up waiting."""
        _check(lib().hm_hmat_check(self.handle, ctypes.c_void_p(_stream_ptr(stream))))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().hm_hmat_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ learned correction

class LearnedCorrection:
    """Learned block-Jacobi correction (hm_lp_*): a per-leaf, per-component scaling of
    the block-Jacobi preconditioner predicted by a small network from leaf features."""

    def __init__(self, theta0=None, hidden=32, handle=None):
        if handle is not None:
            self.handle = handle
            return
        n = lib().hm_lp_param_count(int(hidden))
        if n < 0:
            raise HMError(HM_EINVAL, "hidden width must be 16, 32 or 64")
        th = np.ascontiguousarray(theta0, dtype=np.float64)
        assert th.size == n
        h = ctypes.c_void_p()
        _check(lib().hm_lp_create(int(hidden), th.ctypes.data_as(_VP), ctypes.byref(h)))
        self.handle = h

    @classmethod
    def load(cls, path):
        h = ctypes.c_void_p()
        _check(lib().hm_lp_load(str(path).encode(), ctypes.byref(h)))
        return cls(handle=h)

    def save(self, path):
        _check(lib().hm_lp_save(self.handle, str(path).encode()))

    def info(self):
        i = hm_lp_info()
        _check(lib().hm_lp_get_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in hm_lp_info._fields_}

    def params(self):
        out = np.empty(self.info()["n_params"])
        _check(lib().hm_lp_get_params(self.handle, out.ctypes.data_as(_VP)))
        return out

    def set_fallback(self, on):
        _check(lib().hm_lp_set_fallback(self.handle, 1 if on else 0))

    def set_kind(self, kind, gamma=1.0):
        """kind "scale" (M = D B^-1) or "near" (M = B^-1 - gamma D B^-1 N B^-1)."""
        _check(lib().hm_lp_set_kind(self.handle, {"scale": HM_LP_SCALE, "near": HM_LP_NEAR}[kind], float(gamma)))

    def add_samples(self, features, q):
        f = np.ascontiguousarray(features, dtype=np.float64)
        qq = np.ascontiguousarray(q, dtype=np.float64)
        assert f.shape[1] == 8 and qq.shape == (f.shape[0], 9)
        _check(lib().hm_lp_add_samples(self.handle, f.ctypes.data_as(_VP), qq.ctypes.data_as(_VP), f.shape[0]))

    def add_system(self, H, k, b, x, stream=None):
        """k: float64 CUDA tensor (N,) or None; b, x: float64 CUDA tensors (3N,) or (nrhs, 3N)."""
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        b, x = b.contiguous(), x.contiguous()
        _check(lib().hm_lp_add_system(self.handle, H.handle, _dptr(k) if k is not None else None, _dptr(b),
                                      _dptr(x), int(nrhs), ctypes.c_void_p(_stream_ptr(stream))))

    def clear_samples(self):
        _check(lib().hm_lp_clear_samples(self.handle))

    def loss_grad(self, stream=None):
        g = np.empty(self.info()["n_params"])
        l = ctypes.c_double()
        _check(lib().hm_lp_loss_grad(self.handle, ctypes.byref(l), g.ctypes.data_as(_VP),
                                     ctypes.c_void_p(_stream_ptr(stream))))
        return l.value, g

    def train(self, steps, lr=1e-3, stream=None):
        l = ctypes.c_double()
        _check(lib().hm_lp_train(self.handle, int(steps), float(lr), ctypes.byref(l),
                                 ctypes.c_void_p(_stream_ptr(stream))))
        return l.value

    def predict(self, H, k=None, stream=None):
        """(features (n_leaves x 8), d (n_leaves x 3)) for this H-matrix and k, leaves in cluster order."""
        nl = H.info()["n_leaves"]
        f = np.empty((nl, 8))
        d = np.empty((nl, 3))
        _check(lib().hm_lp_predict(self.handle, H.handle, _dptr(k) if k is not None else None,
                                   f.ctypes.data_as(_VP), d.ctypes.data_as(_VP), ctypes.c_void_p(_stream_ptr(stream))))
        return f, d

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().hm_lp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ autotuner

def autotune_key(el, E, nu, aca_eps, storage, leaves, etas, device, shapes=()):
    """Cache key of a tuning run: the geometry (every element array), the assembly
    options, the candidate list and the device name."""
    import hashlib
    h = hashlib.sha256()
    for k in ("c", "s1", "s2", "n", "a", "b"):
        h.update(np.ascontiguousarray(getattr(el, k), dtype=np.float64).tobytes())
    shape = getattr(el, "shape", None)
    if shape is not None and np.any(np.asarray(shape) != 0):  # triangles: their vertices too
        h.update(np.ascontiguousarray(shape, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(el.tri, dtype=np.float64).tobytes())
    h.update(repr((int(el.N), float(E), float(nu), float(aca_eps), str(storage), tuple(int(v) for v in leaves),
                   tuple(float(v) for v in etas), str(device), tuple(tuple(int(x) for x in t) for t in shapes))).encode())
    return h.hexdigest()[:32]


def autotune(el, E=1.0, nu=0.25, aca_eps=1e-6, storage="f32", leaves=(32, 64, 128), etas=(2.0,), budget_ms=60000,
             cache=None, device=None, stream=None, shapes=None):
    """Fastest (leaf size, eta, tile shape) for the product on this geometry (hm_autotune);
    shapes: (chunk_bytes, chunk_cols, ring, warps) candidates (None: the default shape only).
    With `cache` (a JSON file
    path) a result for the same geometry, options, candidates and device is read from the
    file instead of re-tuning, and new results are added to it."""
    import json
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    shapes = list(shapes) if shapes else []
    key = autotune_key(el, E, nu, aca_eps, storage, leaves, etas, device, shapes)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return table[key]
    ea = _ElemArgs(el)
    st = {"f32": HM_F32, "bf16": HM_BF16, "both": HM_F32_BF16}[storage]
    opt = hm_assemble_opts(float(E), float(nu), float(aca_eps), st, 0, 0.0)
    lv = (_I * len(leaves))(*[int(v) for v in leaves])
    ev = (_D * len(etas))(*[float(v) for v in etas])
    sa = _shape_array(shapes) if shapes else None
    cap = 4096 + 384 * len(leaves) * len(etas) * max(1, len(shapes))
    buf = ctypes.create_string_buffer(cap)
    _check(lib().hm_autotune(ea.ref, ctypes.byref(opt), lv, len(leaves), ev, len(etas), sa, len(shapes),
                             int(budget_ms), buf, cap, ctypes.c_void_p(_stream_ptr(stream))))
    res = json.loads(buf.value.decode())
    res["device"] = device
    if cache:
        table[key] = res
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return res


# ---------------------------------------------------------------- ILU building blocks
def _csr(rowptr, col):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    return rp, cl, int(rp.size - 1)


def ilu_select(i, j, v, p):
    """Indices of the ceil(p n) entries of largest |v| (ties by (i, j)), in that order."""
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty(max(int(np.ceil(p * v.size)), 1) if 0.0 < p <= 1.0 else 1, dtype=np.int64)
    m = ctypes.c_int64()
    _check(lib().hm_ilu_select(int(v.size), i.ctypes.data, j.ctypes.data, v.ctypes.data, float(p),
                               out.ctypes.data, ctypes.byref(m)))
    return out[:m.value]


def ilu_assemble(n, idx, i, j, v, d, order=None):
    """CSR (rowptr, col, val) of the selected entries minus d on the diagonal, renumbered
    by order (new position -> old position) when given."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    od = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    rowptr = np.empty(int(n) + 1, dtype=np.int64)
    cap = max(int(idx.size) + int(n), 1)
    col = np.empty(cap, dtype=np.int32)
    val = np.empty(cap, dtype=np.float64)
    nnz = ctypes.c_int64()
    if not (i.size == j.size == v.size):
        raise HMError(HM_EINVAL, "ilu_assemble: i, j and v must have one length")
    _check(lib().hm_ilu_assemble(int(n), int(v.size), int(idx.size), idx.ctypes.data, i.ctypes.data, j.ctypes.data,
                                 v.ctypes.data, d.ctypes.data, None if od is None else od.ctypes.data,
                                 rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, ctypes.byref(nnz)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def ilu0_factor(rowptr, col, val):
    """ILU(0) of a CSR matrix; returns the factored values (L multipliers and U)."""
    rp, cl, n = _csr(rowptr, col)
    out = np.array(val, dtype=np.float64, copy=True)
    _check(lib().hm_ilu0_factor(n, rp.ctypes.data, cl.ctypes.data, out.ctypes.data))
    return out


def ilu_levels(rowptr, col):
    """(lower levels, upper levels, lower level count, upper level count)."""
    rp, cl, n = _csr(rowptr, col)
    lo = np.empty(max(n, 1), dtype=np.int32)
    up = np.empty(max(n, 1), dtype=np.int32)
    nl, nu = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().hm_ilu_levels(n, rp.ctypes.data, cl.ctypes.data, lo.ctypes.data, up.ctypes.data,
                               ctypes.byref(nl), ctypes.byref(nu)))
    return lo[:n], up[:n], nl.value, nu.value


def ilu_leaf_colours(rowptr, col, leaf_of, n_leaves):
    """(colour of every leaf, colour count)."""
    rp, cl, n = _csr(rowptr, col)
    lf = np.ascontiguousarray(leaf_of, dtype=np.int32)
    out = np.empty(max(int(n_leaves), 1), dtype=np.int32)
    nc = ctypes.c_int32()
    _check(lib().hm_ilu_leaf_colours(n, rp.ctypes.data, cl.ctypes.data, lf.ctypes.data, int(n_leaves),
                                     out.ctypes.data, ctypes.byref(nc)))
    return out[:int(n_leaves)], nc.value


# ---------------------------------------------------------------- interface law
INTERFACE_MODES = ("elastic", "coulomb", "tensile", "open", "apex")


def interface_update(params, T, dp, chi, dd, T1=None, dp1=None, chi1=None, tangent=True, modes=True,
                     counts=False, stream=None):
    """Constitutive update of the interface points and their consistent tangent
    (hm_interface_update).  params: dict or object with Ks, Kn, fp, fr, psip, dc, cp,
    sigp, wc, alphaR; T, dp, chi, dd: (n, 3) FP64 CUDA tensors (T'^n, delta^p, (chi_s,
    chi_t, w_dil), Delta delta).  Outputs default to new tensors (pass the inputs for an
    in-place update).  Returns (T1, dp1, chi1, cep (n, 3, 3) or None, mode (n,) int32 or
    None, counts (6,) int64 numpy or None)."""
    import torch
    n = T.shape[0]
    for a in (T, dp, chi, dd):
        assert a.dtype == torch.float64 and a.is_cuda and a.is_contiguous() and tuple(a.shape) == (n, 3)
    get = (lambda k: params[k]) if isinstance(params, dict) else (lambda k: getattr(params, k))
    prm = hm_interface_params(*[float(get(k)) for k, _ in hm_interface_params._fields_])
    T1 = torch.empty_like(T) if T1 is None else T1
    dp1 = torch.empty_like(dp) if dp1 is None else dp1
    chi1 = torch.empty_like(chi) if chi1 is None else chi1
    cep = torch.empty((n, 3, 3), dtype=torch.float64, device=T.device) if tangent else None
    mode = torch.empty(n, dtype=torch.int32, device=T.device) if modes else None
    cnt = np.zeros(6, dtype=np.int64) if counts else None
    null = ctypes.c_void_p(None)
    _check(lib().hm_interface_update(ctypes.byref(prm), int(n), _dptr(T), _dptr(dp), _dptr(chi), _dptr(dd),
                                     _dptr(T1), _dptr(dp1), _dptr(chi1), _dptr(cep) if tangent else null,
                                     _dptr(mode) if modes else null,
                                     cnt.ctypes.data_as(_P64) if counts else None,
                                     ctypes.c_void_p(_stream_ptr(stream))))
    return T1, dp1, chi1, cep, mode, cnt


# ---------------------------------------------------------------- coupled flow
_PRECONDS = {"none": HM_PRECOND_NONE, "blockj": HM_PRECOND_BLOCKJ, "jacobi3": HM_PRECOND_JACOBI3,
             "ilu": HM_PRECOND_ILU}


class Flow:
    """Fracture flow mesh and matrices (hm_flow_*): conn (N, 4) int32 node indices,
    n_nodes, half sides a, b (N,); for meshes with triangles (linear pressure) also
    shape (N,) and the triangles' vertices tri (N, 9) (hm_flow_create_mesh)."""

    def __init__(self, conn, n_nodes, a, b, shape=None, tri=None):
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        self.N, self.n_nodes = conn.shape[0], int(n_nodes)
        h = ctypes.c_void_p()
        if shape is not None and np.any(np.asarray(shape) != 0):
            sh = np.ascontiguousarray(shape, dtype=np.int32)
            tv = np.ascontiguousarray(tri, dtype=np.float64)
            _check(lib().hm_flow_create_mesh(self.N, sh.ctypes.data_as(_VP), conn.ctypes.data_as(_VP), self.n_nodes,
                                             a.ctypes.data_as(_VP), b.ctypes.data_as(_VP), tv.ctypes.data_as(_VP),
                                             ctypes.byref(h)))
        else:
            _check(lib().hm_flow_create(self.N, conn.ctypes.data_as(_VP), self.n_nodes, a.ctypes.data_as(_VP),
                                        b.ctypes.data_as(_VP), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) is not None and _LIB is not None:
            _LIB.hm_flow_destroy(self.handle)
            self.handle = None

    def assemble(self, params, dn, dp=None, pn=None, stream=None):
        """params: dict with mu, M, w0, dt; dn (N,), dp, pn (n_nodes,) FP64 CUDA tensors."""
        prm = hm_flow_params(*[float(params[k]) for k, _ in hm_flow_params._fields_])
        _check(lib().hm_flow_assemble(self.handle, ctypes.byref(prm), _dptr(dn),
                                      _dptr(dp) if dp is not None else None,
                                      _dptr(pn) if pn is not None else None, ctypes.c_void_p(_stream_ptr(stream))))

    def export(self, stream=None):
        nnz = ctypes.c_int64()
        sp = ctypes.c_void_p(_stream_ptr(stream))
        _check(lib().hm_flow_export(self.handle, ctypes.byref(nnz), None, None, None, None, sp))
        rp = np.empty(self.n_nodes + 1, np.int64)
        col = np.empty(nnz.value, np.int32)
        a22 = np.empty(nnz.value)
        a21 = np.empty((self.N, 4))
        _check(lib().hm_flow_export(self.handle, ctypes.byref(nnz), rp.ctypes.data_as(_P64), col.ctypes.data_as(_VP),
                                    a22.ctypes.data_as(_VP), a21.ctypes.data_as(_VP), sp))
        return dict(rowptr=rp, col=col, a22=a22, a21=a21)

    def matvec(self, H, x, y, k=None, cep=None, shift=0.0, stream=None):
        _check(lib().hm_coupled_matvec(H.handle, self.handle, _dptr(k) if k is not None else None,
                                       _dptr(cep) if cep is not None else None, float(shift), _dptr(x), _dptr(y),
                                       ctypes.c_void_p(_stream_ptr(stream))))

    def solve(self, H, b, x, k=None, cep=None, shift=0.0, tol=1e-8, restart=30, maxit=300, inner_precond="blockj",
              inner_method="fgmres", inner_tol=1e-6, schur_tol=1e-6, ilu_p=0.0, flow_scale=0.0, stream=None,
              raise_on_error=True):
        """Solve the coupled Jacobian system J x = b (hm_coupled_solve); b, x FP64 CUDA
        tensors of length 3N + n_nodes.  Returns the info dict."""
        o = hm_coupled_opts(float(tol), int(restart), int(maxit), _PRECONDS[inner_precond],
                            {"fgmres": HM_METHOD_FGMRES, "bicgstab": HM_METHOD_BICGSTAB}[inner_method],
                            float(inner_tol), float(schur_tol), float(ilu_p), float(flow_scale))
        inf = hm_coupled_info()
        st = lib().hm_coupled_solve(H.handle, self.handle, _dptr(k) if k is not None else None,
                                    _dptr(cep) if cep is not None else None, float(shift), _dptr(b), _dptr(x),
                                    ctypes.byref(o), ctypes.byref(inf), ctypes.c_void_p(_stream_ptr(stream)))
        out = {f: getattr(inf, f) for f, _ in hm_coupled_info._fields_}
        if st != HM_OK and raise_on_error:
            raise HMError(st, lib().hm_last_error().decode())
        return out
