"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.  It shares
no code with the CUDA library (``paper_2605_04497_gb300``): the two meet only at
the seeded inputs from ``synth``.

Every function is a thin ctypes wrapper over ``qts_oracle.c``; the header
``qts_oracle.h`` cites the paper passage each one restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libqts_oracle.so")
_SRC = os.path.join(_HERE, "qts_oracle.c")
_HDR = os.path.join(_HERE, "qts_oracle.h")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -ffp-contract=off so no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Ens(ctypes.Structure):
    _fields_ = [
        ("n_trees", ctypes.c_int32),
        ("n_features", ctypes.c_int32),
        ("node_offsets", ctypes.c_void_p),
        ("left", ctypes.c_void_p),
        ("right", ctypes.c_void_p),
        ("feature", ctypes.c_void_p),
        ("threshold", ctypes.c_void_p),
        ("default_left", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("leaf_value", ctypes.c_void_p),
        ("is_cat", ctypes.c_void_p),
        ("cat_left", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        E = ctypes.POINTER(_Ens)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.orc_gl_nodes.argtypes = [i32, vp, vp]
        lib.orc_predict.argtypes = [E, vp, i64, vp]
        lib.orc_shap_exact.argtypes = [E, vp, i64, i32, vp]
        lib.orc_sii_exact.argtypes = [E, vp, i64, i32, vp, vp]
        lib.orc_shap_quad.argtypes = [E, vp, i64, i32, i32, vp]
        lib.orc_brute_force.argtypes = [E, vp, vp, vp]
        lib.orc_alg1.argtypes = [E, vp, i32, i32, vp]
        lib.orc_grad_exact.argtypes = [E, vp, i64, vp, vp, i64, i32, vp, vp]
        lib.orc_path_stats.argtypes = [E, vp, vp, vp]
        lib.orc_sii3_exact.argtypes = [E, vp, i64, i32, vp]
        lib.orc_brute_force3.argtypes = [E, vp, vp]
        lib.orc_alg1_shap.argtypes = [E, vp, i64, i32, i32, vp]
        lib.orc_sii_order_exact.argtypes = [E, vp, i64, i32, i32, vp]
        lib.orc_brute_force_order.argtypes = [E, vp, i32, vp]
        lib.orc_alg1_order.argtypes = [E, vp, i32, i32, vp]
        for f in ("orc_gl_nodes", "orc_shap_exact", "orc_sii_exact", "orc_shap_quad",
                  "orc_brute_force", "orc_alg1", "orc_grad_exact", "orc_path_stats",
                  "orc_sii3_exact", "orc_brute_force3", "orc_alg1_shap", "orc_sii_order_exact",
                  "orc_brute_force_order", "orc_alg1_order"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return max(1, os.cpu_count() or 1)


class _Bound:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, ens):
        self.arrays = [
            np.ascontiguousarray(ens.node_offsets, dtype=np.int64),
            np.ascontiguousarray(ens.left, dtype=np.int32),
            np.ascontiguousarray(ens.right, dtype=np.int32),
            np.ascontiguousarray(ens.feature, dtype=np.int32),
            np.ascontiguousarray(ens.threshold, dtype=np.float32),
            np.ascontiguousarray(ens.default_left, dtype=np.uint8),
            np.ascontiguousarray(ens.z, dtype=np.float32),
            np.ascontiguousarray(ens.leaf_value, dtype=np.float32),
        ]
        a = self.arrays
        is_cat = getattr(ens, "is_cat", None)
        if is_cat is not None:
            self.arrays += [np.ascontiguousarray(is_cat, dtype=np.uint8),
                            np.ascontiguousarray(ens.cat_left, dtype=np.uint64)]
        cat_ptrs = [x.ctypes.data for x in self.arrays[8:]] if is_cat is not None else [None, None]
        self.s = _Ens(len(a[0]) - 1, int(ens.n_features), *[x.ctypes.data for x in a[:8]], *cat_ptrs)
        self.F = int(ens.n_features)
        self.N = int(a[0][-1])

    def ref(self):
        return ctypes.byref(self.s)


def _f32(X, F):
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2 and X.shape[1] == F, (X.shape, F)
    return X


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed ({rc})")


def gl_nodes(n: int):
    t = np.zeros(n)
    w = np.zeros(n)
    _check(_load().orc_gl_nodes(n, t.ctypes.data, w.ctypes.data), "orc_gl_nodes")
    return t, w


def predict(ens, X) -> np.ndarray:
    b = _Bound(ens)
    X = _f32(X, b.F)
    out = np.zeros(X.shape[0])
    _load().orc_predict(b.ref(), X.ctypes.data, X.shape[0], out.ctypes.data)
    return out


def shap_exact(ens, X, n_threads: int | None = None) -> np.ndarray:
    """phi (M x (F+1)), last column E[f]."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    phi = np.zeros((X.shape[0], b.F + 1))
    _check(_load().orc_shap_exact(b.ref(), X.ctypes.data, X.shape[0], n_threads or threads(),
                                  phi.ctypes.data), "orc_shap_exact")
    return phi


def sii_exact(ens, X, n_threads: int | None = None, with_phi: bool = True):
    """(SII: M x F x F symmetric, zero diagonal, not halved;  phi: M x (F+1))."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    M = X.shape[0]
    sii = np.zeros((M, b.F, b.F))
    phi = np.zeros((M, b.F + 1)) if with_phi else None
    _check(_load().orc_sii_exact(b.ref(), X.ctypes.data, M, n_threads or threads(), sii.ctypes.data,
                                 phi.ctypes.data if with_phi else None), "orc_sii_exact")
    return sii, phi


def interaction_matrix(sii: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Arrange SII and phi in the (F+1) x (F+1) per-sample layout of the
    ``pred_interactions`` convention: off-diagonal SII_ij/2, diagonal
    phi_i - sum_{j!=i} SII_ij/2 (rows sum to phi_i), E[f] at [F, F]."""
    M, F, _ = sii.shape
    out = np.zeros((M, F + 1, F + 1))
    out[:, :F, :F] = sii / 2.0
    idx = np.arange(F)
    out[:, idx, idx] = phi[:, :F] - (sii.sum(axis=2) - sii[:, idx, idx]) / 2.0
    out[:, F, F] = phi[:, F]
    return out


def shap_quad(ens, X, n: int, n_threads: int | None = None) -> np.ndarray:
    b = _Bound(ens)
    X = _f32(X, b.F)
    phi = np.zeros((X.shape[0], b.F + 1))
    _check(_load().orc_shap_quad(b.ref(), X.ctypes.data, X.shape[0], n, n_threads or threads(),
                                 phi.ctypes.data), "orc_shap_quad")
    return phi


def brute_force(ens, x):
    """(phi: F+1, SII: F x F) for one sample by subset enumeration."""
    b = _Bound(ens)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    assert x.shape[0] == b.F
    phi = np.zeros(b.F + 1)
    sii = np.zeros((b.F, b.F))
    _check(_load().orc_brute_force(b.ref(), x.ctypes.data, phi.ctypes.data, sii.ctypes.data),
           "orc_brute_force")
    return phi, sii


def sii3_exact(ens, X, n_threads: int | None = None) -> np.ndarray:
    """Third-order SII: M x F x F x F, symmetric, zero where indices repeat."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    out = np.zeros((X.shape[0], b.F, b.F, b.F))
    _check(_load().orc_sii3_exact(b.ref(), X.ctypes.data, X.shape[0], n_threads or threads(),
                                  out.ctypes.data), "orc_sii3_exact")
    return out


def brute_force3(ens, x) -> np.ndarray:
    b = _Bound(ens)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros((b.F, b.F, b.F))
    _check(_load().orc_brute_force3(b.ref(), x.ctypes.data, out.ctypes.data), "orc_brute_force3")
    return out


def alg1(ens, x, order: int, n: int) -> np.ndarray:
    b = _Bound(ens)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(b.F + 1 if order == 1 else ((b.F, b.F) if order == 2 else (b.F, b.F, b.F)))
    _check(_load().orc_alg1(b.ref(), x.ctypes.data, order, n, out.ctypes.data), "orc_alg1")
    return out


def alg1_shap(ens, X, n: int = 8, n_threads: int | None = None) -> np.ndarray:
    """phi (M x (F+1)) by Algorithm 1 with n Gauss-Legendre points, threaded over
    samples; at most min(n_threads, M) threads run."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    phi = np.zeros((X.shape[0], b.F + 1))
    _check(_load().orc_alg1_shap(b.ref(), X.ctypes.data, X.shape[0], n, n_threads or threads(),
                                 phi.ctypes.data), "orc_alg1_shap")
    return phi


def n_subsets(F: int, s: int) -> int:
    from math import comb

    return comb(F, s)


def sii_order_exact(ens, X, s: int, n_threads: int | None = None) -> np.ndarray:
    """Order-s SII, M x C(F, s), subsets in lexicographic order."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    out = np.zeros((X.shape[0], n_subsets(b.F, s)))
    _check(_load().orc_sii_order_exact(b.ref(), X.ctypes.data, X.shape[0], s, n_threads or threads(),
                                       out.ctypes.data), "orc_sii_order_exact")
    return out


def brute_force_order(ens, x, s: int) -> np.ndarray:
    b = _Bound(ens)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(n_subsets(b.F, s))
    _check(_load().orc_brute_force_order(b.ref(), x.ctypes.data, s, out.ctypes.data), "orc_brute_force_order")
    return out


def alg1_order(ens, x, s: int, n: int) -> np.ndarray:
    b = _Bound(ens)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(n_subsets(b.F, s))
    _check(_load().orc_alg1_order(b.ref(), x.ctypes.data, s, n, out.ctypes.data), "orc_alg1_order")
    return out


def grad_exact(ens, X, grad_phi, leaves=None, n_threads: int | None = None):
    """(d_leaf, d_z), each of length N (nodes), of L = sum grad_phi * phi."""
    b = _Bound(ens)
    X = _f32(X, b.F)
    G = np.ascontiguousarray(grad_phi, dtype=np.float32)
    assert G.shape == (X.shape[0], b.F + 1)
    d_leaf = np.zeros(b.N)
    d_z = np.zeros(b.N)
    if leaves is not None:
        leaves = np.ascontiguousarray(leaves, dtype=np.int64)
    _check(_load().orc_grad_exact(b.ref(), X.ctypes.data, X.shape[0], G.ctypes.data,
                                  leaves.ctypes.data if leaves is not None else None,
                                  0 if leaves is None else len(leaves), n_threads or threads(),
                                  d_leaf.ctypes.data, d_z.ctypes.data), "orc_grad_exact")
    return d_leaf, d_z


def path_stats(ens):
    b = _Bound(ens)
    n = np.zeros(1, dtype=np.int64)
    d = np.zeros(1, dtype=np.int32)
    s = np.zeros(1, dtype=np.int64)
    _check(_load().orc_path_stats(b.ref(), n.ctypes.data, d.ctypes.data, s.ctypes.data),
           "orc_path_stats")
    return int(n[0]), int(d[0]), int(s[0])
