"""Compile the plain-C brute-force checker (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "naive_knn.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libnaive_knn.so")


def build(force: bool = False) -> str:
    """gcc -O2 -ffp-contract=off: products are never fused into adds, so the
    binary64 arithmetic follows the definition on x86-64 and aarch64 alike."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.naive_knn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.naive_knn.restype = None
        lib.naive_cosine.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.naive_cosine.restype = ctypes.c_double
        _lib = lib
    return _lib


def naive_knn(x: np.ndarray, q: np.ndarray, k: int):
    """Run the C brute force: returns (idx int64[nq,k], dist, score)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    nq, f = q.shape
    idx = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float64)
    score = np.empty((nq, k), dtype=np.float64)
    lib.naive_knn(x.ctypes.data, x.shape[0], f, q.ctypes.data, nq, k,
                  idx.ctypes.data, dist.ctypes.data, score.ctypes.data)
    return idx, dist, score


def naive_cosine(q: np.ndarray, x: np.ndarray) -> float:
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    return lib.naive_cosine(q.ctypes.data, x.ctypes.data, q.shape[0])
