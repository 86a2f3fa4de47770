"""ctypes loader for oracle.c (FP64 gridding loops and direct back-projection).

TEST INFRASTRUCTURE ONLY: compiled with gcc on first use (or by the build
step), never linked into the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    so = os.path.join(_HERE, "_oracle.so")
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp, "-lm"])
    os.replace(tmp, so)
    return so


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.orc_spread2d.argtypes = [ctypes.c_long, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            L.orc_spread1d.argtypes = [ctypes.c_long, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _dp]
            L.orc_bpa.argtypes = [ctypes.c_int] * 4 + [_dp] * 5 + [ctypes.c_long, _dp, _dp]
            for f in (L.orc_spread2d, L.orc_spread1d, L.orc_bpa):
                f.restype = None
            _LIB = L
    return _LIB


def _p(a):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def spread2d(x, y, c, Mrx, Mry, w, taux, tauy, G):
    assert c.dtype == np.complex128 and G.dtype == np.complex128
    lib().orc_spread2d(x.size, c.shape[1], _p(x), _p(y), _p(c), Mrx, Mry, w, taux, tauy, _p(G))


def spread1d(t, c, Mr, w, tau, g):
    assert c.dtype == np.complex128 and g.dtype == np.complex128
    lib().orc_spread1d(c.shape[0], c.shape[1], _p(t), _p(c), Mr, w, tau, _p(g))


def bpa(echo, pos, tx, rx, freq, vox):
    echo = np.ascontiguousarray(echo, np.complex128)
    T, R, P, Nk = echo.shape
    vox = np.ascontiguousarray(vox, np.float64).reshape(-1, 3)
    out = np.zeros(vox.shape[0], np.complex128)
    lib().orc_bpa(T, R, P, Nk, _p(np.ascontiguousarray(pos, np.float64)), _p(np.ascontiguousarray(tx, np.float64)),
                  _p(np.ascontiguousarray(rx, np.float64)), _p(np.ascontiguousarray(freq, np.float64)), _p(echo),
                  vox.shape[0], _p(vox), _p(out))
    return out
