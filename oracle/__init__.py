"""FP64 CPU oracle for arbitrary-shape-surface Fresnel diffraction (Eq. 7).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1203_3583_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``asfd_oracle.c`` (plain C, FP64, OpenMP over
destination points); this module compiles it with gcc and marshals numpy
arrays through ctypes.  ``eq7`` is the direct O(N^2) per-point sum of the
discretised Eq. 7 (Sec. 2); ``eq7_grad`` writes out the derivative of that sum
with respect to the source field and the height map.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asfd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libasfd_oracle.so")
_lock = threading.Lock()
_lib = None


class Geom(ctypes.Structure):
    """Mirror of ``asfd_oracle_geom`` (oracle-private; not the library's struct)."""

    _fields_ = [
        ("n1x", ctypes.c_int), ("n1y", ctypes.c_int),
        ("p1x", ctypes.c_double), ("p1y", ctypes.c_double),
        ("m2x", ctypes.c_int), ("m2y", ctypes.c_int),
        ("p2x", ctypes.c_double), ("p2y", ctypes.c_double),
        ("lam", ctypes.c_double), ("z0", ctypes.c_double),
        ("sx", ctypes.c_double), ("sy", ctypes.c_double),
        ("ox", ctypes.c_double), ("oy", ctypes.c_double),
    ]


def compile_c(src: str, out: str) -> str:
    """gcc -O2 -fopenmp shared build of one oracle C source (IEEE FP64, no contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libasfd_oracle.so`` (and the 1D
    oracle of ``oracle/line.py`` beside it)."""
    os.makedirs(_BUILD, exist_ok=True)
    from . import line
    line.build(force)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_c(_SRC, _LIB_PATH)


def bind(path: str):
    """Load a compiled oracle library from `path` and declare its signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.asfd_oracle_eq7.argtypes = [ctypes.POINTER(Geom), dp, dp, ctypes.c_int,
                                    ip, ip, dp, ctypes.c_int]
    lib.asfd_oracle_eq7.restype = ctypes.c_int
    for name in ("asfd_oracle_eq5", "asfd_oracle_eq2"):
        fn = getattr(lib, name)
        fn.argtypes = lib.asfd_oracle_eq7.argtypes
        fn.restype = ctypes.c_int
    lib.asfd_oracle_eq7_grad.argtypes = [ctypes.POINTER(Geom), dp, dp, ctypes.c_int,
                                         ip, ip, dp, dp, dp, ctypes.c_int]
    lib.asfd_oracle_eq7_grad.restype = ctypes.c_int
    lib.asfd_oracle_max_threads.argtypes = []
    lib.asfd_oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def max_threads() -> int:
    """OpenMP threads the oracle uses by default (all host cores)."""
    return int(_load().asfd_oracle_max_threads())


def _geom(g: dict) -> Geom:
    for key in ("n1x", "n1y", "m2x", "m2y"):
        if int(g[key]) <= 0 or int(g[key]) % 2:
            raise ValueError(f"{key} must be a positive even integer")
    return Geom(int(g["n1x"]), int(g["n1y"]), float(g["p1x"]), float(g["p1y"]),
                int(g["m2x"]), int(g["m2y"]), float(g["p2x"]), float(g["p2y"]),
                float(g["lam"]), float(g["z0"]), float(g.get("sx", 0.0)), float(g.get("sy", 0.0)),
                float(g.get("ox", 0.0)), float(g.get("oy", 0.0)))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _points(g: dict, points):
    if points is None:
        my, mx = np.meshgrid(np.arange(g["m2y"]), np.arange(g["m2x"]), indexing="ij")
        return np.ascontiguousarray(mx.ravel(), np.int32), np.ascontiguousarray(my.ravel(), np.int32)
    mx, my = points
    return np.ascontiguousarray(mx, np.int32), np.ascontiguousarray(my, np.int32)


def eq7(g: dict, u1: np.ndarray, d1: np.ndarray, points=None, nthreads: int = 0,
        lib=None) -> np.ndarray:
    """Discretised Eq. 7 at destination points.

    g: dict with n1x, n1y, p1x, p1y, m2x, m2y, p2x, p2y, lam, z0 (SI units).
    u1: complex [n1y, n1x]; d1: real [n1y, n1x] (metres, toward the destination).
    points: None for the full [m2y, m2x] grid, else (mx, my) integer arrays.
    Returns complex128 of shape [m2y, m2x] (full grid) or [len(mx)].
    """
    gg = _geom(g)
    u1c = np.ascontiguousarray(u1, np.complex128)
    d1c = np.ascontiguousarray(d1, np.float64)
    if u1c.shape != (gg.n1y, gg.n1x) or d1c.shape != (gg.n1y, gg.n1x):
        raise ValueError("u1 and d1 must have shape (n1y, n1x)")
    mx, my = _points(g, points)
    out = np.empty(mx.size, np.complex128)
    rc = (lib or _load()).asfd_oracle_eq7(ctypes.byref(gg), _dptr(u1c.view(np.float64)), _dptr(d1c),
                                 int(mx.size), _iptr(mx), _iptr(my),
                                 _dptr(out.view(np.float64)), int(nthreads))
    if rc != 0:
        raise RuntimeError("asfd_oracle_eq7 rejected its arguments")
    if points is None:
        return out.reshape(gg.m2y, gg.m2x)
    return out


def _direct(name: str, g: dict, u1, d1, points, nthreads, lib):
    gg = _geom(g)
    u1c = np.ascontiguousarray(u1, np.complex128)
    d1c = np.ascontiguousarray(d1, np.float64)
    if u1c.shape != (gg.n1y, gg.n1x) or d1c.shape != (gg.n1y, gg.n1x):
        raise ValueError("u1 and d1 must have shape (n1y, n1x)")
    mx, my = _points(g, points)
    out = np.empty(mx.size, np.complex128)
    rc = getattr(lib or _load(), name)(ctypes.byref(gg), _dptr(u1c.view(np.float64)), _dptr(d1c),
                                       int(mx.size), _iptr(mx), _iptr(my),
                                       _dptr(out.view(np.float64)), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"{name} rejected its arguments")
    return out.reshape(gg.m2y, gg.m2x) if points is None else out


def eq5(g: dict, u1: np.ndarray, d1: np.ndarray, points=None, nthreads: int = 0,
        lib=None) -> np.ndarray:
    """Eq. 5 (per-sample r0 in the destination chirp) at destination points;
    arguments and result as for eq7."""
    return _direct("asfd_oracle_eq5", g, u1, d1, points, nthreads, lib)


def eq2(g: dict, u1: np.ndarray, d1: np.ndarray, points=None, nthreads: int = 0,
        lib=None) -> np.ndarray:
    """Eq. 2 (Huygens sum with the exact distance of Eq. 3) at destination
    points; arguments and result as for eq7."""
    return _direct("asfd_oracle_eq2", g, u1, d1, points, nthreads, lib)


def eq7_grad(g: dict, u1: np.ndarray, d1: np.ndarray, gu2: np.ndarray, points=None,
             nthreads: int = 0, lib=None):
    """Gradients (dL/du1 as complex, dL/dd1 as real) of a real loss through Eq. 7.

    gu2 holds dL/dRe(u2) + i dL/dIm(u2) at the destination points (full grid
    [m2y, m2x] when points is None).  Returns (gu1 [n1y, n1x] complex,
    gd1 [n1y, n1x] real).
    """
    gg = _geom(g)
    u1c = np.ascontiguousarray(u1, np.complex128)
    d1c = np.ascontiguousarray(d1, np.float64)
    mx, my = _points(g, points)
    gu2c = np.ascontiguousarray(np.asarray(gu2).ravel(), np.complex128)
    if gu2c.size != mx.size:
        raise ValueError("gu2 must have one value per destination point")
    gu1 = np.empty((gg.n1y, gg.n1x), np.complex128)
    gd1 = np.empty((gg.n1y, gg.n1x), np.float64)
    rc = (lib or _load()).asfd_oracle_eq7_grad(ctypes.byref(gg), _dptr(u1c.view(np.float64)), _dptr(d1c),
                                      int(mx.size), _iptr(mx), _iptr(my),
                                      _dptr(gu2c.view(np.float64)),
                                      _dptr(gu1.view(np.float64)), _dptr(gd1), int(nthreads))
    if rc != 0:
        raise RuntimeError("asfd_oracle_eq7_grad rejected its arguments")
    return gu1, gd1
