"""CPU FP64 stencil oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it.

``gather`` advances a grid by the gather-mode definition (Eq. (stencil-2d9p),
generalised to d = 2, 3 and order r); ``sample`` returns single output points
computed on their dependency cones.  Both run the C code in
``stencil_oracle.c`` (plain multiply-then-add in FP64, lexicographic term
order).  See that file's header for the boundary conventions.

``min_line_cover`` is the minimal set of axis-parallel coefficient lines of a
2D weight pattern (Sec. 3.5), found by trying every set of row lines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

_BC = {"dirichlet": 0, "periodic": 1}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc (OpenMP if available)."""
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(_SRC):
        return LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_gather.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int,
                                          ctypes.c_int64, dp, dp]
            lib.oracle_gather.restype = ctypes.c_int
            lib.oracle_sample.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int,
                                          ctypes.c_int64, dp, ctypes.c_int64, i64p, dp,
                                          ctypes.c_int64]
            lib.oracle_sample.restype = ctypes.c_int
            lib.oracle_threads.argtypes = []
            lib.oracle_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _check(r, coeffs, ndim):
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.shape != (2 * r + 1,) * ndim:
        raise ValueError(f"coeffs shape {c.shape} does not match r={r}, ndim={ndim}")
    return c


def gather(field: np.ndarray, r: int, coeffs: np.ndarray, bc: str, steps: int) -> np.ndarray:
    """Advance ``field`` (float64, C order, interior points) by ``steps`` sweeps."""
    lib = _load()
    a = np.ascontiguousarray(field, dtype=np.float64)
    ndim = a.ndim
    c = _check(r, coeffs, ndim)
    shape = np.array(a.shape, dtype=np.int64)
    out = np.empty_like(a)
    rc = lib.oracle_gather(ndim, _ip(shape), r, _dp(c), _BC[bc], int(steps), _dp(a), _dp(out))
    if rc != 0:
        raise RuntimeError(f"oracle_gather failed with code {rc}")
    return out


def sample(field: np.ndarray, r: int, coeffs: np.ndarray, bc: str, steps: int,
           points: np.ndarray, max_window: int = 1 << 27) -> np.ndarray:
    """Output values at ``points`` (int array [npts, ndim]) after ``steps`` sweeps."""
    lib = _load()
    a = np.ascontiguousarray(field, dtype=np.float64)
    ndim = a.ndim
    c = _check(r, coeffs, ndim)
    pts = np.ascontiguousarray(points, dtype=np.int64).reshape(-1, ndim)
    shape = np.array(a.shape, dtype=np.int64)
    vals = np.empty(pts.shape[0], dtype=np.float64)
    rc = lib.oracle_sample(ndim, _ip(shape), r, _dp(c), _BC[bc], int(steps), _dp(a),
                           pts.shape[0], _ip(pts), _dp(vals), int(max_window))
    if rc != 0:
        raise RuntimeError(f"oracle_sample failed with code {rc}")
    return vals


def threads() -> int:
    """Number of host threads the oracle uses."""
    return int(_load().oracle_threads())


def error_norms(got: np.ndarray, ref: np.ndarray):
    """(rel_l2, rel_max) of ``got`` against ``ref``, in float64."""
    g = np.asarray(got, dtype=np.float64).ravel()
    o = np.asarray(ref, dtype=np.float64).ravel()
    d = g - o
    nref = np.sqrt(np.dot(o, o))
    mref = np.max(np.abs(o)) if o.size else 0.0
    rel_l2 = float(np.sqrt(np.dot(d, d)) / nref) if nref > 0 else float(np.sqrt(np.dot(d, d)))
    rel_max = float(np.max(np.abs(d)) / mref) if mref > 0 else float(np.max(np.abs(d), initial=0.0))
    return rel_l2, rel_max


def min_line_cover(mask):
    """Minimal axis-parallel line cover of a 2D weight pattern (Sec. 3.5).

    ``mask`` is an n x n array whose nonzero entries mark the weights present.
    A cover is a set of row lines and column lines such that every nonzero
    (i, j) lies on row i or on column j of the set.  Brute force over every
    set of row lines: once the rows are fixed, the columns that must be added
    are exactly those holding a nonzero in a row left out.  Returns
    (number of lines, rows, cols) for one minimal cover, rows and cols as
    boolean arrays; among minimal covers the first one met is returned (row
    sets in increasing binary order).  Exponential in n: small n only.
    """
    m = np.asarray(mask) != 0
    n = m.shape[0]
    if m.ndim != 2 or m.shape[1] != n:
        raise ValueError("mask must be square")
    if n > 16:
        raise ValueError("brute force is for n <= 16")
    best = None
    for bits in range(1 << n):
        rows = np.array([(bits >> i) & 1 for i in range(n)], dtype=bool)
        cols = np.zeros(n, dtype=bool)
        for i in range(n):
            if not rows[i]:
                for j in range(n):
                    if m[i, j]:
                        cols[j] = True
        count = int(rows.sum() + cols.sum())
        if best is None or count < best[0]:
            best = (count, rows, cols)
    return best
