"""Oracle — test infrastructure only (tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does).

Python front end of `direct.c`: the sparse Fourier transform by its definition,
eq. 1.1 (Sec. 1), u_i = sum_j exp(2 pi i x_i.k_j / N) f_j, in FP64 on the host cores,
and its adjoint f_j = sum_i exp(-2 pi i x_i.k_j / N) u_i.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_oracle_direct.so")
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Builds oracle/_oracle_direct.so with gcc and OpenMP (portable flags, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_oracle())
        lib.oracle_direct.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int]
        lib.oracle_direct.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_threads())


def _direct(x, k, f, N, sign, nthreads):
    x = np.ascontiguousarray(x, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.float64)
    if x.ndim != 2 or k.ndim != 2 or x.shape[1] != k.shape[1]:
        raise ValueError("x and k must be [n, dim] with the same dim")
    f = np.asarray(f)
    squeeze = f.ndim == 1
    f2 = np.ascontiguousarray(np.atleast_2d(f), dtype=np.complex128)
    if f2.shape[1] != k.shape[0]:
        raise ValueError("f must have one entry per source point")
    nrhs = f2.shape[0]
    u = np.zeros((nrhs, x.shape[0]), dtype=np.complex128)
    if x.shape[0] and k.shape[0]:
        _load().oracle_direct(x.shape[1], float(N), x.shape[0], x.ctypes.data, k.shape[0],
                              k.ctypes.data, nrhs, f2.ctypes.data, u.ctypes.data, sign,
                              int(nthreads))
    return u[0] if squeeze else u


def direct(x, k, f, N, nthreads: int = 0):
    """u_i = sum_j exp(+2 pi i x_i.k_j/N) f_j (eq. 1.1).  f: [nk] or [nrhs, nk] complex."""
    return _direct(x, k, f, N, +1, nthreads)


def direct_adjoint(x, k, u, N, nthreads: int = 0):
    """f_j = sum_i exp(-2 pi i x_i.k_j/N) u_i, the conjugate transpose of eq. 1.1."""
    return _direct(k, x, u, N, -1, nthreads)
