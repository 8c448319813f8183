"""ctypes loader of the multi-threaded C FP64 oracle (``spmttkrp_ref.c``), used for timing.

TEST INFRASTRUCTURE ONLY (tests, smoke check, the benchmark's CPU legs).  ``build()``
compiles it in-tree with the host C compiler, OpenMP when available, and without
floating-point contraction so that its results equal the NumPy oracle bit for bit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmttkrp_ref.c")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liboracle_ref.so")

_lib = None


def build() -> str:
    """Compiles the C oracle if the library is missing or older than its source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP: the same code, one thread
        subprocess.run(base, check=True)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.spm_oracle_mttkrp.restype = ctypes.c_int
        _lib.spm_oracle_threads.restype = ctypes.c_int
    return _lib


def threads() -> int:
    return int(lib().spm_oracle_threads())


def mttkrp(coo, vals, dims, factors, n, nthreads=0):
    """Mode-n spMTTKRP in FP64 (same result as ``oracle.mttkrp``), on nthreads host threads
    (0 = all)."""
    coo = np.ascontiguousarray(np.asarray(coo, dtype=np.int64))
    vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    F = [np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in factors]
    N = coo.shape[1]
    R = F[0].shape[1]
    if not 0 <= n < N or len(F) != N or dims.shape[0] != N:
        raise ValueError("mode, factors or dims do not match the coordinates")
    out = np.zeros((int(dims[n]), R), dtype=np.float64)
    fp = (ctypes.c_void_p * N)(*[f.ctypes.data for f in F])
    st = lib().spm_oracle_mttkrp(
        ctypes.c_void_p(coo.ctypes.data), ctypes.c_void_p(vals.ctypes.data),
        ctypes.c_int64(coo.shape[0]), ctypes.c_int(N), ctypes.c_void_p(dims.ctypes.data), fp,
        ctypes.c_int(R), ctypes.c_int(n), ctypes.c_void_p(out.ctypes.data), ctypes.c_int(nthreads))
    if st != 0:
        raise ValueError("C oracle rejected its arguments")
    return out
