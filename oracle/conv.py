"""FP64 oracle of the surrogate's 3-D convolutions (forward, backward-data,
backward-weight), channels-last.  TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "conv3d_oracle.c")
_LIB = os.path.join(_HERE, "libconv_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", _SRC, "-o",
                        tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            L.oracle_conv3d_fwd.argtypes = [dp, dp, dp, dp, i, i, i, i, i, i, i]
            L.oracle_conv3d_bwd_data.argtypes = [dp, dp, dp, i, i, i, i, i, i, i]
            L.oracle_conv3d_bwd_weight.argtypes = [dp, dp, dp, dp, i, i, i, i, i, i, i]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def conv3d_fwd(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """x [N,D,H,W,Ci], w [Co,k,k,k,Ci], b [Co] -> y [N,D,H,W,Co]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N, D, H, W, Ci = x.shape
    Co, k = w.shape[0], w.shape[1]
    y = np.zeros((N, D, H, W, Co))
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    lib().oracle_conv3d_fwd(_p(x), _p(w), _p(bb), _p(y), N, D, H, W, Ci, Co, k)
    return y


def conv3d_bwd_data(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N, D, H, W, Co = dy.shape
    k, Ci = w.shape[1], w.shape[4]
    dx = np.zeros((N, D, H, W, Ci))
    lib().oracle_conv3d_bwd_data(_p(dy), _p(w), _p(dx), N, D, H, W, Ci, Co, k)
    return dx


def conv3d_bwd_weight(x: np.ndarray, dy: np.ndarray, k: int):
    x = np.ascontiguousarray(x, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    N, D, H, W, Ci = x.shape
    Co = dy.shape[4]
    dw = np.zeros((Co, k, k, k, Ci))
    db = np.zeros(Co)
    lib().oracle_conv3d_bwd_weight(_p(x), _p(dy), _p(dw), _p(db), N, D, H, W, Ci, Co, k)
    return dw, db
