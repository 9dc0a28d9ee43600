"""The oracle: a plain, slow FP64 CPU restatement of the sDEM total viewshed.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2003_02200_gb300``) never imports, links or calls it, and the two share
no code.  See ``tvs_oracle.c`` for what is computed and which passages of the
paper each step follows (Alg. 1-4 for the problem, section 4.1 and Alg. 6-9 for
the sampling, walk and interpolation rules).

The C source is compiled on first use with gcc into ``liboracle.so`` next to
this file (``-O2 -fopenmp -ffp-contract=off``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcDir(C.Structure):
    _fields_ = [
        ("frame", C.c_int), ("m", C.c_int), ("H", C.c_int), ("W", C.c_int),
        ("t_fx", C.c_uint64), ("t", C.c_double), ("g", C.c_double),
        ("K", C.c_int64), ("D", C.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into liboracle.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i64p = C.POINTER(C.c_int64)
            f64p = C.POINTER(C.c_double)
            lib.orc_direction.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.POINTER(OrcDir)]
            lib.orc_total_viewshed.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.POINTER(C.c_int), i64p]
            lib.orc_cell_direction.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), i64p, f64p, i64p, i64p]
            lib.orc_line_cv.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                C.c_int, C.c_int64, C.c_void_p, C.c_int]
            lib.orc_line_range.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, i64p, i64p]
            lib.orc_column_offsets.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                               C.c_void_p, C.c_int]
            lib.orc_direct_viewshed.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                C.c_void_p, C.c_int64, C.c_void_p]
            lib.orc_visibility_map.argtypes = [
                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                C.c_void_p, C.c_int, C.c_void_p]
            lib.orc_count_evals.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
            lib.orc_count_evals.restype = C.c_int64
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _dem(dem) -> np.ndarray:
    a = np.ascontiguousarray(dem, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("dem must be 2-D")
    return a


def direction(n: int, k: int, rows: int, cols: int, step: float = 1.0, max_range: float = 0.0) -> dict:
    d = OrcDir()
    _check(load().orc_direction(n, k, rows, cols, step, max_range, C.byref(d)), "direction")
    return {f: getattr(d, f) for f, _ in OrcDir._fields_}


def total_viewshed(dem, step: float, h0: float, n: int, max_range: float = 0.0, prec: int = 64,
                   cells=None, nthreads: int = 0, info: dict | None = None) -> np.ndarray:
    """Visible area (squared units of step) per cell; cells = flat indices or None for all."""
    a = _dem(dem)
    rows, cols = a.shape
    if cells is None:
        idx_p, count = None, rows * cols
    else:
        idx = np.ascontiguousarray(cells, dtype=np.int64)
        idx_p, count = idx.ctypes.data, idx.size
    out = np.empty(count, dtype=np.float64)
    used = C.c_int(0)
    nev = C.c_int64(0)
    _check(load().orc_total_viewshed(a.ctypes.data, rows, cols, step, h0, n, max_range, prec,
                                     idx_p, count, out.ctypes.data, nthreads, C.byref(used),
                                     C.byref(nev)), "total_viewshed")
    if info is not None:
        info["threads"] = used.value
        info["evals_visited"] = nev.value
    return out.reshape(rows, cols) if cells is None else out


def direct_viewshed(dem, step: float, h0: float, n: int, max_range: float = 0.0, prec: int = 64,
                    cells=None) -> np.ndarray:
    """Singular viewsheds by definition (Alg. 1-3: lines of sight through the
    POV cell itself, no virtual POVs) of the cells listed by flat index."""
    a = _dem(dem)
    idx = np.ascontiguousarray(cells, dtype=np.int64).ravel()
    out = np.empty(idx.size, dtype=np.float64)
    _check(load().orc_direct_viewshed(a.ctypes.data, a.shape[0], a.shape[1], step, h0, n, max_range, prec,
                                      idx.ctypes.data, idx.size, out.ctypes.data), "direct_viewshed")
    return out


def visibility_map(dem, step: float, h0: float, n: int, max_range: float = 0.0, prec: int = 64,
                   povs=((0, 0),)) -> np.ndarray:
    """Number of the POVs (row, col) that see each cell (int32 map)."""
    a = _dem(dem)
    p = np.ascontiguousarray(povs, dtype=np.int32).reshape(-1, 2)
    count = np.zeros(a.shape, dtype=np.int32)
    _check(load().orc_visibility_map(a.ctypes.data, a.shape[0], a.shape[1], step, h0, n, max_range, prec,
                                     p.ctypes.data, len(p), count.ctypes.data), "visibility_map")
    return count


def cell_direction(dem, step, h0, n, max_range, prec, i, j, k) -> list[dict]:
    a = _dem(dem)
    rows, cols = a.shape
    npov = C.c_int(0)
    b = (C.c_int64 * 2)()
    w = (C.c_double * 2)()
    cf = (C.c_int64 * 2)()
    cb = (C.c_int64 * 2)()
    _check(load().orc_cell_direction(a.ctypes.data, rows, cols, step, h0, n, max_range, prec, i, j, k,
                                     C.byref(npov), b, w, cf, cb), "cell_direction")
    return [dict(b=b[v], w=w[v], cv_fwd=cf[v], cv_bwd=cb[v]) for v in range(npov.value)]


def line_cv(dem, step, h0, n, max_range, prec, k, b) -> np.ndarray:
    a = _dem(dem)
    rows, cols = a.shape
    W = max(rows, cols)
    out = np.empty(W, dtype=np.int64)
    _check(load().orc_line_cv(a.ctypes.data, rows, cols, step, h0, n, max_range, prec, k, b,
                              out.ctypes.data, W), "line_cv")
    d = direction(n, k, rows, cols)
    return out[: d["W"]]


def line_range(n, k, rows, cols, b) -> tuple[int, int]:
    lo = C.c_int64(0)
    hi = C.c_int64(0)
    _check(load().orc_line_range(n, k, rows, cols, b, C.byref(lo), C.byref(hi)), "line_range")
    return lo.value, hi.value


def column_offsets(n, k, rows, cols) -> tuple[np.ndarray, np.ndarray]:
    W = max(rows, cols)
    dest = np.empty(W, dtype=np.int64)
    frac = np.empty(W, dtype=np.uint32)
    _check(load().orc_column_offsets(n, k, rows, cols, dest.ctypes.data, frac.ctypes.data, W),
           "column_offsets")
    Wk = direction(n, k, rows, cols)["W"]
    return dest[:Wk], frac[:Wk]


def count_evals(rows, cols, n, step=1.0, max_range=0.0) -> int:
    E = load().orc_count_evals(rows, cols, n, step, max_range)
    if E < 0:
        raise ValueError("count_evals failed")
    return int(E)
