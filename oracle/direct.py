"""O_direct: the exact product y = A x of Eq. (1) by a plain double loop.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The arithmetic lives in
oracle/direct.c (FP64, one sequential sum per row); this module only loads it.
"""
import ctypes

import numpy as np

from ._build import build_oracle

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.oracle_direct_rows.restype = None
        lib.oracle_direct_rows.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p]
        lib.oracle_direct_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def direct_rows(targets, sources, kappa, x, rows=None):
    """Rows `rows` of A x with A[j,k] = exp(i kappa r)/(4 pi r), r = |x_j - y_k|.

    targets: (N_T, 3) float64, sources: (N_S, 3) float64, x: (N_S,) complex128.
    Coincident target/source pairs contribute 0 (zero diagonal, Sect. 4).
    Returns complex128 array of len(rows) (all rows when rows is None).
    """
    lib = _load()
    t = np.ascontiguousarray(targets, dtype=np.float64)
    s = np.ascontiguousarray(sources, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.complex128)
    if rows is None:
        rows = np.arange(t.shape[0], dtype=np.int64)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros(r.shape[0], dtype=np.complex128)
    lib.oracle_direct_rows(t.ctypes.data, t.shape[0], s.ctypes.data,
                           s.shape[0], float(kappa), xv.ctypes.data,
                           r.ctypes.data, r.shape[0], y.ctypes.data)
    return y


def direct_threads():
    """OpenMP threads the direct sum runs on."""
    return int(_load().oracle_direct_threads())
