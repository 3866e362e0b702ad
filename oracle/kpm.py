"""ctypes front end of kpm_oracle.c (test infrastructure only).

Follows Algorithm 1, Eq. 3term and the Appendix A doubling identity; see the
C file's header for the passages and the one sign correction.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB_PATH, build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = LIB_PATH if os.path.exists(LIB_PATH) else build_oracle()
        L = C.CDLL(path)
        L.oracle_splitmix64_next.restype = C.c_uint64
        L.oracle_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.oracle_rademacher.restype = C.c_double
        L.oracle_rademacher.argtypes = [C.c_uint64] * 4
        L.oracle_start_block.restype = None
        L.oracle_start_block.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_uint64,
                                         C.c_uint64, C.c_void_p]
        L.oracle_kpm_moments.restype = C.c_int
        L.oracle_kpm_moments.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_double, C.c_double, C.c_int, C.c_int64,
                                         C.c_int64, C.c_uint64, C.c_uint64, C.c_int,
                                         C.c_int, C.c_int, C.c_void_p]
        L.oracle_gershgorin.restype = None
        L.oracle_gershgorin.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.oracle_spmv.restype = None
        L.oracle_spmv.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
        L.oracle_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _csr_arrays(row_ptr, col_idx, val):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)  # FP32 values are upcast exactly
    return rp, ci, va


def splitmix64_stream(seed: int, count: int) -> list[int]:
    st = C.c_uint64(seed)
    return [int(lib().oracle_splitmix64_next(C.byref(st))) for _ in range(count)]


def rademacher(seed: int, b: int, l: int, i: int) -> float:
    return float(lib().oracle_rademacher(seed, b, l, i))


def start_block(n: int, n_v: int, seed: int, batch_index: int = 0, vec_offset: int = 0) -> np.ndarray:
    """Start vectors as an (n, n_v) array (row i, column l)."""
    out = np.empty((n, n_v), dtype=np.float64)
    lib().oracle_start_block(n, n_v, vec_offset, seed, batch_index, out.ctypes.data)
    return out


_MODES = {"direct": 0, "doubling": 1, "legendre": 2}


def kpm_moments_per_vector(A, lb: float, ub: float, M: int, n_v: int, seed: int, *,
                           mode: str = "doubling", batch_index: int = 0, vec_offset: int = 0,
                           reverse: bool = False, nthreads: int = 0) -> np.ndarray:
    """mu_k^(l) = v_l^T T_k(B) v_l / n, shape (n_v, M+1), B = (A - cI)/d."""
    rp, ci, va = _csr_arrays(A.row_ptr, A.col_idx, A.val)
    out = np.empty((n_v, M + 1), dtype=np.float64)
    rc = lib().oracle_kpm_moments(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                                  float(lb), float(ub), int(M), int(n_v), int(vec_offset),
                                  int(seed), int(batch_index), _MODES[mode],
                                  1 if reverse else 0, int(nthreads), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_kpm_moments rejected its arguments")
    return out


def kpm_moments(A, lb, ub, M, n_v, seed, **kw) -> np.ndarray:
    """mu_k = (1/(n n_v)) sum_l v_l^T T_k(B) v_l, k = 0..M."""
    return kpm_moments_per_vector(A, lb, ub, M, n_v, seed, **kw).mean(axis=0)


def spmv(A, x: np.ndarray) -> np.ndarray:
    rp, ci, va = _csr_arrays(A.row_ptr, A.col_idx, A.val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    lib().oracle_spmv(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, x.ctypes.data,
                      y.ctypes.data)
    return y


def num_threads() -> int:
    return int(lib().oracle_num_threads())
