"""FP64 CPU oracle of the one-dimensional form with explicit source samples
(``asfd_oracle_line.c``): Eq. 7, Eq. 5 or Eq. 2 on a line source sampled at
arbitrary positions x1 with heights d1 and weights w.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import compile_c

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asfd_oracle_line.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libasfd_oracle_line.so")
_lock = threading.Lock()
_lib = None


class LineGeom(ctypes.Structure):
    """Mirror of ``asfd_oracle_line_geom``."""

    _fields_ = [("m2", ctypes.c_int), ("p2", ctypes.c_double), ("lam", ctypes.c_double),
                ("z0", ctypes.c_double), ("s", ctypes.c_double)]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_c(_SRC, _LIB_PATH)


def bind(path: str):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.asfd_oracle_line.argtypes = [ctypes.POINTER(LineGeom), dp, dp, dp, dp, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int]
    lib.asfd_oracle_line.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
        return _lib


def line(g: dict, x1, d1, w, u1, form: int = 7, points=None, nthreads: int = 0,
         lib=None) -> np.ndarray:
    """1D Eq. 7 / 5 / 2 (form) at destination indices `points` (default: all m2).

    g: dict with m2, p2, lam, z0 and optional s (incidence direction cosine).
    x1, d1, w: real [n] (metres); u1: complex [n].  Returns complex128 [npts].
    """
    gg = LineGeom(int(g["m2"]), float(g["p2"]), float(g["lam"]), float(g["z0"]),
                  float(g.get("s", 0.0)))
    x1c = np.ascontiguousarray(x1, np.float64)
    d1c = np.ascontiguousarray(d1, np.float64)
    wc = np.ascontiguousarray(w, np.float64)
    u1c = np.ascontiguousarray(u1, np.complex128)
    n = x1c.size
    if not (d1c.size == wc.size == u1c.size == n):
        raise ValueError("x1, d1, w and u1 must have the same length")
    m = (np.arange(gg.m2, dtype=np.int32) if points is None
         else np.ascontiguousarray(points, np.int32))
    out = np.empty(m.size, np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = (lib or _load()).asfd_oracle_line(
        ctypes.byref(gg), x1c.ctypes.data_as(dp), d1c.ctypes.data_as(dp), wc.ctypes.data_as(dp),
        u1c.view(np.float64).ctypes.data_as(dp), int(n), int(form), int(m.size),
        m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.view(np.float64).ctypes.data_as(dp),
        int(nthreads))
    if rc != 0:
        raise RuntimeError("asfd_oracle_line rejected its arguments")
    return out
