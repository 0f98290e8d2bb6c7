"""Python binding of libqtreeshap (GB300 Quadrature-TreeSHAP).

Thin ctypes marshalling over the C ABI declared in ``include/qtreeshap.h``;
every step of the computation runs in the library's CUDA kernels.  PyTorch is
used only for device memory and streams.  If the shared library has not been
built (``__graft_entry__.build()`` or ``python paper_2605_04497_gb300/build.py``)
importing the compute functions raises - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqtreeshap.so")

QTS_OK = 0
QTS_FLAG_FP64 = 1
QTS_DESCRIBE_PAIRS = 2
# n_quad = EXACT_NODES: per path width w the fewest Gauss-Legendre points that
# integrate an order-s quantity exactly, ceil((w - s + 1) / 2) (Thm 2)
EXACT_NODES = 0
STATUS_NAMES = {0: "QTS_OK", 1: "QTS_ERR_ARG", 2: "QTS_ERR_CUDA", 3: "QTS_ERR_OOM",
                4: "QTS_ERR_UNSUPPORTED", 5: "QTS_ERR_TIMEOUT", 6: "QTS_ERR_DEVICE_CHECK"}

# every symbol include/qtreeshap.h declares
EXPORTS = ("qts_load_ensemble", "qts_load_ensemble_cat", "qts_update_params", "qts_shap_values", "qts_shap_values_alg1",
           "qts_shap_interactions",
           "qts_shap_interactions_noalloc", "qts_shap_interactions3", "qts_shap_interactions_order",
           "qts_shap_backward", "qts_batched_fwd_bwd", "qts_batched_autotune", "qts_get_batch_info", "qts_autotune", "qts_sync_status",
           "qts_get_info", "qts_describe_ensemble", "qts_describe_paths", "qts_describe_alg1_program", "qts_selftest_wait_timeout", "qts_batched_kernel_count", "qts_batched_last_kernel_ms", "qts_gauss_legendre", "qts_exact_nodes", "qts_fp32_pipe_peak", "qts_last_error",
           "qts_free")

_lib = None


class QtsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class QtsInfo(ctypes.Structure):
    _fields_ = [
        ("n_trees", ctypes.c_int32), ("n_features", ctypes.c_int32),
        ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("n_paths", ctypes.c_int64),
        ("max_unique", ctypes.c_int32), ("sum_unique", ctypes.c_int64),
        ("n_buckets", ctypes.c_int32), ("bucket_width", ctypes.c_int32 * 32),
        ("bucket_paths", ctypes.c_int64 * 32), ("expected_value", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("flags", ctypes.c_uint32),
    ]


class QtsRequest(ctypes.Structure):
    _fields_ = [
        ("ens", ctypes.c_void_p), ("X", ctypes.c_void_p), ("M", ctypes.c_int64),
        ("F", ctypes.c_int32), ("grad_phi", ctypes.c_void_p), ("phi", ctypes.c_void_p),
        ("d_leaf", ctypes.c_void_p), ("d_z", ctypes.c_void_p),
    ]


def lib():
    """Load the shared library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        L.qts_load_ensemble.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, u32,
                                        ctypes.POINTER(vp)]
        L.qts_load_ensemble_cat.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, u32,
                                            ctypes.POINTER(ctypes.c_void_p)]
        L.qts_update_params.argtypes = [vp, vp, vp]
        L.qts_shap_values.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.qts_shap_values_alg1.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.qts_shap_interactions.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.qts_shap_interactions_noalloc.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.qts_shap_interactions3.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.qts_shap_interactions_order.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp]
        L.qts_shap_backward.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, vp]
        L.qts_batched_fwd_bwd.argtypes = [i32, vp, i32, vp]
        L.qts_batched_autotune.argtypes = [i32, vp, i32, i64, vp, vp]
        L.qts_get_batch_info.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.qts_autotune.argtypes = [vp, vp, i64, i32, ctypes.c_char_p, vp]
        L.qts_sync_status.argtypes = [vp, vp]
        L.qts_selftest_wait_timeout.argtypes = [vp, vp]
        L.qts_get_info.argtypes = [vp, ctypes.POINTER(QtsInfo)]
        L.qts_describe_ensemble.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, u32,
                                            ctypes.POINTER(QtsInfo)]
        L.qts_gauss_legendre.argtypes = [i32, vp, vp]
        L.qts_exact_nodes.argtypes = [i32, i32]
        L.qts_fp32_pipe_peak.argtypes = [i32, vp, vp]
        L.qts_describe_alg1_program.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
        L.qts_describe_paths.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]
        L.qts_batched_kernel_count.argtypes = []
        L.qts_batched_last_kernel_ms.argtypes = [ctypes.POINTER(ctypes.c_float)]
        L.qts_last_error.argtypes = []
        L.qts_last_error.restype = ctypes.c_char_p
        L.qts_free.argtypes = [vp]
        L.qts_free.restype = None
        for f in EXPORTS:
            if f not in ("qts_last_error", "qts_free", "qts_batched_kernel_count", "qts_exact_nodes"):
                getattr(L, f).restype = ctypes.c_int
        L.qts_batched_kernel_count.restype = ctypes.c_int32
        L.qts_exact_nodes.restype = ctypes.c_int32
        _lib = L
    return _lib


def _check(status: int):
    if status != QTS_OK:
        raise QtsError(status, lib().qts_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def gauss_legendre(n: int):
    t = np.zeros(n)
    w = np.zeros(n)
    _check(lib().qts_gauss_legendre(n, t.ctypes.data, w.ctypes.data))
    return t, w


def fp32_pipe_peak(packed: bool = True, stream=None) -> float:
    """Measured FP32-pipe throughput in lane FMAs per second (an f32x2 FMA
    counts two)."""
    v = ctypes.c_double()
    _check(lib().qts_fp32_pipe_peak(1 if packed else 0, ctypes.byref(v), _stream(stream)))
    return v.value


def exact_nodes(width: int, order: int = 1) -> int:
    """Points n_quad = EXACT_NODES takes on paths of `width` unique features
    for an order-`order` quantity (0 for arguments out of range)."""
    return int(lib().qts_exact_nodes(width, order))


def _info_dict(i: QtsInfo) -> dict:
    nb = i.n_buckets
    return dict(n_trees=i.n_trees, n_features=i.n_features, n_nodes=i.n_nodes,
                n_leaves=i.n_leaves, n_paths=i.n_paths, max_unique=i.max_unique,
                sum_unique=i.sum_unique, buckets=list(zip(i.bucket_width[:nb], i.bucket_paths[:nb])),
                expected_value=i.expected_value, device_bytes=i.device_bytes, flags=i.flags)


def describe(ens, fp64: bool = False, pairs: bool = False) -> dict:
    """Host-only path preparation summary (no GPU needed); pairs: the tables of
    the batched pass (sibling leaves merged)."""
    arr = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
    a = [arr(ens.node_offsets, np.int64), arr(ens.left, np.int32), arr(ens.right, np.int32),
         arr(ens.feature, np.int32), arr(ens.threshold, np.float32), arr(ens.default_left, np.uint8),
         arr(ens.z, np.float32), arr(ens.leaf_value, np.float32)]
    i = QtsInfo()
    flags = (QTS_FLAG_FP64 if fp64 else 0) | (QTS_DESCRIBE_PAIRS if pairs else 0)
    _check(lib().qts_describe_ensemble(len(a[0]) - 1, *[x.ctypes.data for x in a], int(ens.n_features),
                                       flags, ctypes.byref(i)))
    return _info_dict(i)


def describe_paths(ens) -> dict:
    """Host-only: the FP32 path tables the library would upload (records as
    n_records x 4 uint32 bit patterns, each path's leaf and bucket width)."""
    arr = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
    a = [arr(ens.node_offsets, np.int64), arr(ens.left, np.int32), arr(ens.right, np.int32),
         arr(ens.feature, np.int32), arr(ens.threshold, np.float32), arr(ens.default_left, np.uint8),
         arr(ens.z, np.float32), arr(ens.leaf_value, np.float32)]
    is_cat = getattr(ens, "is_cat", None)
    cat = [arr(is_cat, np.uint8), arr(ens.cat_left, np.uint64)] if is_cat is not None else None
    cat_ptrs = [c.ctypes.data for c in cat] if cat else [None, None]
    n_rec, n_path = ctypes.c_int64(), ctypes.c_int64()
    args = [len(a[0]) - 1, *[x.ctypes.data for x in a], *cat_ptrs, int(ens.n_features),
            ctypes.byref(n_rec), ctypes.byref(n_path)]
    _check(lib().qts_describe_paths(*args, None, None, None))
    rec = np.zeros((n_rec.value, 4), np.uint32)
    leaf = np.zeros(n_path.value, np.int64)
    width = np.zeros(n_path.value, np.int32)
    _check(lib().qts_describe_paths(*args, rec.ctypes.data, leaf.ctypes.data, width.ctypes.data))
    return dict(records=rec, path_leaf=leaf, path_width=width)


def describe_alg1_program(ens) -> dict:
    """Host-only: the preorder record program of the depth-first form (records
    as n_records x 8 uint32 bit patterns, per-tree offsets, stack levels)."""
    arr = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
    a = [arr(ens.node_offsets, np.int64), arr(ens.left, np.int32), arr(ens.right, np.int32),
         arr(ens.feature, np.int32), arr(ens.threshold, np.float32), arr(ens.default_left, np.uint8),
         arr(ens.z, np.float32), arr(ens.leaf_value, np.float32)]
    n = ctypes.c_int64()
    args = [len(a[0]) - 1, *[x.ctypes.data for x in a], int(ens.n_features), ctypes.byref(n)]
    _check(lib().qts_describe_alg1_program(*args, None, None, None))
    rec = np.zeros((n.value, 8), np.uint32)
    off = np.zeros(len(a[0]), np.int64)
    levels = ctypes.c_int32()
    _check(lib().qts_describe_alg1_program(*args, rec.ctypes.data, off.ctypes.data, ctypes.byref(levels)))
    return dict(records=rec, tree_off=off, levels=levels.value)


class Ensemble:
    """A tree ensemble loaded into device path tables (owns the C handle)."""

    def __init__(self, node_offsets, left, right, feature, threshold, default_left, z, leaf_value,
                 n_features: int, fp64: bool = False, is_cat=None, cat_left=None):
        arr = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        self._off = arr(node_offsets, np.int64)
        self._host = dict(left=arr(left, np.int32), right=arr(right, np.int32),
                          feature=arr(feature, np.int32), threshold=arr(threshold, np.float32),
                          default_left=arr(default_left, np.uint8), z=arr(z, np.float32),
                          leaf_value=arr(leaf_value, np.float32))
        self.n_features = int(n_features)
        self.n_trees = len(self._off) - 1
        self.n_nodes = int(self._off[-1])
        self.fp64 = bool(fp64)
        h = ctypes.c_void_p()
        H = self._host
        common = [self.n_trees, self._off.ctypes.data, H["left"].ctypes.data, H["right"].ctypes.data,
                  H["feature"].ctypes.data, H["threshold"].ctypes.data, H["default_left"].ctypes.data,
                  H["z"].ctypes.data, H["leaf_value"].ctypes.data]
        flags = QTS_FLAG_FP64 if fp64 else 0
        if is_cat is None:
            _check(lib().qts_load_ensemble(*common, self.n_features, flags, ctypes.byref(h)))
        else:
            H["is_cat"] = arr(is_cat, np.uint8)
            H["cat_left"] = arr(cat_left, np.uint64)
            _check(lib().qts_load_ensemble_cat(*common, H["is_cat"].ctypes.data, H["cat_left"].ctypes.data,
                                               self.n_features, flags, ctypes.byref(h)))
        self.handle = h

    @classmethod
    def from_arrays(cls, ens, fp64: bool = False) -> "Ensemble":
        """From any object with node_offsets/left/right/feature/threshold/
        default_left/z/leaf_value/n_features attributes."""
        return cls(ens.node_offsets, ens.left, ens.right, ens.feature, ens.threshold,
                   ens.default_left, ens.z, ens.leaf_value, ens.n_features, fp64=fp64,
                   is_cat=getattr(ens, "is_cat", None), cat_left=getattr(ens, "cat_left", None))

    def update_params(self, z, leaf_value):
        z = np.ascontiguousarray(z, dtype=np.float32)
        lv = np.ascontiguousarray(leaf_value, dtype=np.float32)
        assert z.shape == (self.n_nodes,) and lv.shape == (self.n_nodes,)
        _check(lib().qts_update_params(self.handle, z.ctypes.data, lv.ctypes.data))
        self._host["z"], self._host["leaf_value"] = z, lv

    def info(self) -> dict:
        i = QtsInfo()
        _check(lib().qts_get_info(self.handle, ctypes.byref(i)))
        return _info_dict(i)

    def batch_info(self) -> dict:
        """Sizes of the tables the batched pass uses (sibling leaf pairs merged)."""
        n, su, npair = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        nb = ctypes.c_int32()
        bw = (ctypes.c_int32 * 32)()
        bp = (ctypes.c_int64 * 32)()
        _check(lib().qts_get_batch_info(self.handle, ctypes.byref(n), ctypes.byref(su), ctypes.byref(npair),
                                        ctypes.byref(nb), bw, bp))
        return dict(n_paths=n.value, sum_unique=su.value, n_pair_paths=npair.value,
                    buckets=[(int(bw[i]), int(bp[i])) for i in range(nb.value)])

    def sync_status(self, stream=None):
        _check(lib().qts_sync_status(self.handle, _stream(stream)))

    def selftest_wait_timeout(self, stream=None):
        """Enqueue a bounded wait that runs out (about a second); the next
        sync_status raises QtsError with QTS_ERR_TIMEOUT."""
        _check(lib().qts_selftest_wait_timeout(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().qts_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_x(ens: Ensemble, X):
    import torch

    assert isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32, "X: cuda float32"
    assert X.dim() == 2 and X.shape[1] == ens.n_features and X.is_contiguous(), "X: M x F contiguous"


def shap_values(ens: Ensemble, X, n_quad: int = 8, out=None, stream=None):
    """phi (M x (F+1), float64, last column E[f]) on X's device."""
    import torch

    _check_x(ens, X)
    M, F = X.shape
    if out is None:
        out = torch.empty((M, F + 1), dtype=torch.float64, device=X.device)
    _check(lib().qts_shap_values(ens.handle, _ptr(X), M, F, n_quad, _ptr(out), _stream(stream)))
    return out


def shap_values_alg1(ens: Ensemble, X, n_quad: int = 8, out=None, stream=None):
    """Like shap_values, computed by the depth-first traversal of Algorithm 1."""
    import torch

    _check_x(ens, X)
    M, F = X.shape
    if out is None:
        out = torch.empty((M, F + 1), dtype=torch.float64, device=X.device)
    _check(lib().qts_shap_values_alg1(ens.handle, _ptr(X), M, F, n_quad, _ptr(out), _stream(stream)))
    return out


def shap_interactions(ens: Ensemble, X, n_quad: int = 8, out=None, stream=None):
    """M x (F+1) x (F+1) float32: off-diagonal SII/2, diagonal phi_i - row sum, E[f] at [F,F]."""
    import torch

    _check_x(ens, X)
    M, F = X.shape
    if out is None:
        out = torch.empty((M, F + 1, F + 1), dtype=torch.float32, device=X.device)
    _check(lib().qts_shap_interactions(ens.handle, _ptr(X), M, F, n_quad, _ptr(out),
                                       _stream(stream)))
    return out


def shap_interactions_noalloc(ens: Ensemble, X, out, n_quad: int = 8, stream=None):
    """Like shap_interactions, for callers that must not allocate device memory
    during the call: `out` (M x (F+1) x (F+1) float32) is caller-provided and the
    library's fixed 16 MiB scratch holds the accumulators (see the C header for
    the size limit and the no-overlap rule)."""
    _check_x(ens, X)
    M, F = X.shape
    _check(lib().qts_shap_interactions_noalloc(ens.handle, _ptr(X), M, F, n_quad, _ptr(out),
                                               _stream(stream)))
    return out


def triple_index(F: int):
    """Compact index of each triple a < b < c (the layout of shap_interactions3)."""
    from math import comb

    idx = {}
    for a in range(F):
        for b in range(a + 1, F):
            for c in range(b + 1, F):
                idx[(a, b, c)] = (comb(F, 3) - comb(F - a, 3)) + (comb(F - a - 1, 2) - comb(F - b, 2)) + (c - b - 1)
    return idx


def shap_interactions3(ens: Ensemble, X, n_quad: int = 8, out=None, stream=None):
    """Third-order SII, compact: M x C(F,3) float32 over triples a < b < c."""
    import torch
    from math import comb

    _check_x(ens, X)
    M, F = X.shape
    if out is None:
        out = torch.empty((M, comb(F, 3)), dtype=torch.float32, device=X.device)
    _check(lib().qts_shap_interactions3(ens.handle, _ptr(X), M, F, n_quad, _ptr(out), _stream(stream)))
    return out


def shap_interactions_order(ens: Ensemble, X, order: int, n_quad: int = 8, out=None, stream=None):
    """M x C(F, order) float32: SII of every feature subset of size `order`,
    subsets in lexicographic order (itertools.combinations(range(F), order))."""
    import math

    import torch

    _check_x(ens, X)
    M, F = X.shape
    if out is None:
        out = torch.empty((M, math.comb(F, order)), dtype=torch.float32, device=X.device)
    _check(lib().qts_shap_interactions_order(ens.handle, _ptr(X), M, F, order, n_quad, _ptr(out),
                                             _stream(stream)))
    return out


def expand_triples(compact, F: int):
    """Dense symmetric M x F x F x F array (numpy) from the compact layout."""
    c = np.asarray(compact)
    out = np.zeros((c.shape[0], F, F, F), dtype=c.dtype)
    for (a, b, cc), t in triple_index(F).items():
        v = c[:, t]
        for i, j, k in ((a, b, cc), (a, cc, b), (b, a, cc), (b, cc, a), (cc, a, b), (cc, b, a)):
            out[:, i, j, k] = v
    return out


def shap_backward(ens: Ensemble, X, grad_phi, n_quad: int = 8, stream=None, d_leaf=None, d_z=None):
    """(d_leaf, d_z), float64 of length n_nodes: gradients of sum(grad_phi * phi).
    Pass d_leaf / d_z to write into existing tensors."""
    import torch

    _check_x(ens, X)
    M, F = X.shape
    assert grad_phi.shape == (M, F + 1) and grad_phi.dtype == torch.float32 and grad_phi.is_contiguous()
    if d_leaf is None:
        d_leaf = torch.empty(ens.n_nodes, dtype=torch.float64, device=X.device)
    if d_z is None:
        d_z = torch.empty(ens.n_nodes, dtype=torch.float64, device=X.device)
    for t in (d_leaf, d_z):
        assert t.shape == (ens.n_nodes,) and t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    _check(lib().qts_shap_backward(ens.handle, _ptr(X), M, F, n_quad, _ptr(grad_phi), _ptr(d_leaf),
                                   _ptr(d_z), _stream(stream)))
    return d_leaf, d_z


def make_requests(items):
    """items: list of dicts with ens, X, grad_phi (optional), phi, d_leaf, d_z tensors."""
    reqs = (QtsRequest * len(items))()
    for r, it in zip(reqs, items):
        X = it["X"]
        r.ens = it["ens"].handle.value
        r.X = X.data_ptr()
        r.M = X.shape[0]
        r.F = X.shape[1]
        r.grad_phi = it["grad_phi"].data_ptr() if it.get("grad_phi") is not None else 0
        r.phi = it["phi"].data_ptr() if it.get("phi") is not None else 0
        r.d_leaf = it["d_leaf"].data_ptr() if it.get("d_leaf") is not None else 0
        r.d_z = it["d_z"].data_ptr() if it.get("d_z") is not None else 0
    return reqs


def batched_fwd_bwd(reqs, n_quad: int = 8, stream=None):
    """Run prepared ``make_requests`` in one persistent launch (graph-captured)."""
    _check(lib().qts_batched_fwd_bwd(len(reqs), ctypes.cast(reqs, ctypes.c_void_p), n_quad,
                                     _stream(stream)))


def batched_autotune(reqs, n_quad: int = 8, max_samples: int = 1024, stream=None) -> dict:
    """Tune the batched launch for these requests (see qts_batched_autotune);
    returns {width: (paths per item, sample mapping, blocks per SM or 0)} for
    the tuned widths."""
    n = 65  # QTS_MAX_UNIQUE_FEATURES_PER_PATH + 1
    chosen = np.zeros(3 * n, dtype=np.int32)
    _check(lib().qts_batched_autotune(len(reqs), ctypes.cast(reqs, ctypes.c_void_p), n_quad, max_samples,
                                      chosen.ctypes.data, _stream(stream)))
    return {D: (int(chosen[3 * D]), int(chosen[3 * D + 1]), int(chosen[3 * D + 2]))
            for D in range(n) if chosen[3 * D] > 0}


def batched_last_kernel_ms() -> float:
    """Device time of the persistent kernel of this thread's last batched call."""
    ms = ctypes.c_float()
    _check(lib().qts_batched_last_kernel_ms(ctypes.byref(ms)))
    return float(ms.value)


def batched_kernel_count() -> int:
    return int(lib().qts_batched_kernel_count())


def autotune(ens: Ensemble, X, cache_path: str | None = None, stream=None):
    _check_x(ens, X)
    M, F = X.shape
    _check(lib().qts_autotune(ens.handle, _ptr(X), M, F,
                              cache_path.encode() if cache_path else None, _stream(stream)))


class QTreeShapFn:
    """torch.autograd.Function: phi = QTreeShap(leaf_values, z; X).

    ``leaf_values`` and ``z`` are float32 tensors of length n_nodes (the
    ensemble's parameters); backward returns dL/d leaf_values and dL/d z from the
    adjoint kernel (float64 results cast to the parameters' dtype)."""

    _fn = None

    @classmethod
    def apply(cls, ens: Ensemble, leaf_values, z, X, n_quad: int = 8):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, leaf_values, z, X, ens, n_quad):
                    lv = leaf_values.detach().cpu().numpy()
                    zz = z.detach().cpu().numpy()
                    if not (np.array_equal(lv, ens._host["leaf_value"]) and
                            np.array_equal(zz, ens._host["z"])):
                        ens.update_params(zz, lv)
                    ctx.ens, ctx.n_quad = ens, n_quad
                    ctx.dev_l, ctx.dev_z = leaf_values.device, z.device
                    ctx.dt_l, ctx.dt_z = leaf_values.dtype, z.dtype
                    ctx.save_for_backward(X)
                    return shap_values(ens, X, n_quad)

                @staticmethod
                def backward(ctx, grad_phi):
                    (X,) = ctx.saved_tensors
                    g = grad_phi.to(torch.float32).contiguous()
                    d_leaf, d_z = shap_backward(ctx.ens, X, g, ctx.n_quad)
                    return (d_leaf.to(device=ctx.dev_l, dtype=ctx.dt_l),
                            d_z.to(device=ctx.dev_z, dtype=ctx.dt_z), None, None, None)

            cls._fn = _F
        return cls._fn.apply(leaf_values, z, X, ens, n_quad)
