"""The oracle's sparse apply y = A x on all host cores (OpenMP C), beside scipy's one-thread product.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

``build()`` compiles csr_spmv.c with gcc into oracle/_build/; ``CsrSpmv(A)`` holds an assembled
scipy CSR matrix with 64-bit indices and applies it with a chosen number of threads.  Every row is
summed in column order, as scipy does, so the result equals scipy's product bit for bit.
Pinned by: equality with scipy's product (tests/test_oracle_spmv.py).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcsr_spmv.so")


def build() -> str:
    src = os.path.join(HERE, "csr_spmv.c")
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
    subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB, src], check=True)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.oracle_csr_spmv.argtypes = [ctypes.c_int64, p, p, p, p, p]
        lib.oracle_csr_spmv.restype = None
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


class CsrSpmv:
    """y = A x for one assembled CSR matrix, with `threads` OpenMP threads."""

    def __init__(self, A):
        A = A.tocsr()
        self.n = A.shape[0]
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int64)
        self.data = np.ascontiguousarray(A.data, dtype=np.float64)

    def __call__(self, x: np.ndarray, threads: int | None = None) -> np.ndarray:
        lib = _load()
        if threads is not None:
            lib.oracle_set_threads(int(threads))
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        lib.oracle_csr_spmv(self.n, self.indptr.ctypes.data, self.indices.ctypes.data, self.data.ctypes.data,
                            x.ctypes.data, y.ctypes.data)
        return y
