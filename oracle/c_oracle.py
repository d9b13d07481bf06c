"""ctypes loader for the C version of O1 (TEST INFRASTRUCTURE).

``build()`` compiles ``exact_cgemm.c`` with gcc (-O2, OpenMP) into
``liboracle_exact.so`` next to it.  The same source builds on x86-64 and on
aarch64: it uses only ``unsigned __int128`` and portable C.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exact_cgemm.c")
_LIB = os.path.join(_HERE, "liboracle_exact.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_cgemm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     P, P, P, P, P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int]
        lib.oracle_cgemm.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return _load().oracle_max_threads()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rounded_cgemm(A, B, p: int, entries=None, nthreads: int = 0):
    """RN_p(A B) (4M definition).  With ``entries`` (array of (i, j)), only those.

    Returns (sign[2, N], exp[2, N], limb[2, L, N]) with N = m*n (row-major)
    or len(entries).
    """
    lib = _load()
    m, k, n = A.rows, A.cols, B.cols
    L = (p + 63) // 64
    if A.limb.shape[1] != L or B.limb.shape[1] != L:
        raise ValueError("limb count does not match p")
    Asg, Aex, Ali = (np.ascontiguousarray(x) for x in (A.sign, A.exp, A.limb))
    Bsg, Bex, Bli = (np.ascontiguousarray(x) for x in (B.sign, B.exp, B.limb))
    if entries is not None:
        ent = np.ascontiguousarray(np.asarray(entries, dtype=np.int64).reshape(-1, 2))
        total = ent.shape[0]
        eptr = _ptr(ent)
    else:
        ent = None
        total = m * n
        eptr = None
    sg = np.zeros((2, total), np.uint8)
    ex = np.zeros((2, total), np.int32)
    li = np.zeros((2, L, total), np.uint64)
    rc = lib.oracle_cgemm(m, n, k, p, _ptr(Asg), _ptr(Aex), _ptr(Ali), _ptr(Bsg), _ptr(Bex),
                          _ptr(Bli), eptr, total, _ptr(sg), _ptr(ex), _ptr(li), int(nthreads))
    if rc == -34:
        from .exact import ExponentRangeError
        raise ExponentRangeError("result exponent outside int32")
    if rc != 0:
        raise RuntimeError(f"oracle_cgemm failed: {rc}")
    return sg, ex, li


def rounded_cgemm_matrix(A, B, p: int, nthreads: int = 0):
    """Full product as an ``MPCMatrix`` (all m*n entries)."""
    from synthetic_inputs import MPCMatrix
    m, n = A.rows, B.cols
    sg, ex, li = rounded_cgemm(A, B, p, None, nthreads)
    L = li.shape[1]
    return MPCMatrix(m, n, p, sg.reshape(2, m, n), ex.reshape(2, m, n), li.reshape(2, L, m, n))
