"""ctypes wrapper around the FP64 C oracle (test infrastructure only).

Grids and radars are the dataclasses of the ``synth`` package; arrays are numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grft_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Radar(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("fc", C.c_double), ("prf", C.c_double),
                ("dr", C.c_double), ("c", C.c_double)]


def build(force: bool = False) -> str:
    """Compile grft_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = C.CDLL(path)
            P = C.c_void_p
            i32, f64 = C.c_int32, C.c_double
            R = C.POINTER(_Radar)
            lib.orc_num_threads.restype = C.c_int
            lib.orc_bins_phases.argtypes = [R, P, P, C.c_int, P, P]
            lib.orc_grft_plain_rows.argtypes = [R, P, i32, i32, f64, f64, f64, f64, P, P, C.c_int, P,
                                                C.c_int]
            lib.orc_coarse_rm.argtypes = [R, P, i32, i32, f64, f64, i32, f64, f64, i32, i32, i32, P,
                                          C.c_int]
            lib.orc_dsgrft_rows.argtypes = [R, P, i32, i32, f64, f64, i32, f64, f64, i32, i32, i32, P,
                                            P, C.c_int, P, C.c_int]
            lib.orc_cfar_detect.argtypes = [P, i32, i32, i32, i32, i32, f64, f64, i32, i32, P, P,
                                            C.c_int]
            lib.orc_cfar_detect.restype = C.c_long
            lib.orc_trajectory_grad.argtypes = [R, P, i32, P, i32, P, P, P, P, P, C.c_int]
            lib.orc_refine.argtypes = [R, P, i32, P, P, i32, i32, P, C.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(load().orc_num_threads())


def _radar(r) -> _Radar:
    return _Radar(r.M, r.N, r.fc_hz, r.prf_hz, r.dr_m, r.c_mps)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _echo(s: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.complex64)
    return s


def bins_phases(radar, v, a):
    """rho[h][m] int32 and w[h][m] complex128 for explicit (v, a) pairs."""
    v = np.ascontiguousarray(v, dtype=np.float64).ravel()
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    nh = v.size
    rho = np.zeros((nh, radar.M), dtype=np.int32)
    w = np.zeros((nh, radar.M), dtype=np.complex128)
    R = _radar(radar)
    load().orc_bins_phases(C.byref(R), _p(v), _p(a), nh, _p(rho), _p(w))
    return rho, w


def grft_plain_rows(radar, s, grid, vi, ai, nthreads: int = 0) -> np.ndarray:
    """Y[row][n0] complex128 for plain-grid rows (vi[row], ai[row])."""
    s = _echo(s)
    vi = np.ascontiguousarray(vi, dtype=np.int32).ravel()
    ai = np.ascontiguousarray(ai, dtype=np.int32).ravel()
    Y = np.zeros((vi.size, grid.r0_count), dtype=np.complex128)
    R = _radar(radar)
    load().orc_grft_plain_rows(C.byref(R), _p(s), grid.r0_begin, grid.r0_count, grid.v.start,
                               grid.v.step, grid.a.start, grid.a.step, _p(vi), _p(ai), vi.size,
                               _p(Y), nthreads)
    return Y


def grft_plain_full(radar, s, grid, nthreads: int = 0) -> np.ndarray:
    """Y[v][a][n0] complex128 over the whole plain grid."""
    vi, ai = np.meshgrid(np.arange(grid.v.count), np.arange(grid.a.count), indexing="ij")
    Y = grft_plain_rows(radar, s, grid, vi.ravel(), ai.ravel(), nthreads)
    return Y.reshape(grid.v.count, grid.a.count, grid.r0_count)


def coarse_rm(radar, s, ds, cell_begin: int, cell_count: int, nthreads: int = 0) -> np.ndarray:
    """Z[cell][m][n0] complex128 (time-domain mGIFT)."""
    s = _echo(s)
    Z = np.zeros((cell_count, radar.M, ds.r0_count), dtype=np.complex128)
    R = _radar(radar)
    load().orc_coarse_rm(C.byref(R), _p(s), ds.r0_begin, ds.r0_count, ds.vc.start, ds.vc.step,
                         ds.vc.count, ds.ac.start, ds.ac.step, ds.ac.count, cell_begin, cell_count,
                         _p(Z), nthreads)
    return Z


def dsgrft_rows(radar, s, ds, cell, fine, nthreads: int = 0) -> np.ndarray:
    """Y[row][n0] complex128 for DS rows (cell[row], fine[row]), fine = k*Fa + q."""
    s = _echo(s)
    cell = np.ascontiguousarray(cell, dtype=np.int32).ravel()
    fine = np.ascontiguousarray(fine, dtype=np.int32).ravel()
    Y = np.zeros((cell.size, ds.r0_count), dtype=np.complex128)
    R = _radar(radar)
    load().orc_dsgrft_rows(C.byref(R), _p(s), ds.r0_begin, ds.r0_count, ds.vc.start, ds.vc.step,
                           ds.vc.count, ds.ac.start, ds.ac.step, ds.ac.count, ds.Fv, ds.Fa,
                           _p(cell), _p(fine), cell.size, _p(Y), nthreads)
    return Y


def ds_rows_of_canonical(ds, v_full, a_full):
    """Map canonical indices v_full = i*Fv + k, a_full = l*Fa + q to (cell, fine)."""
    v_full = np.asarray(v_full)
    a_full = np.asarray(a_full)
    i, k = v_full // ds.Fv, v_full % ds.Fv
    l, q = a_full // ds.Fa, a_full % ds.Fa
    return i * ds.ac.count + l, k * ds.Fa + q


def dsgrft_full(radar, s, ds, nthreads: int = 0) -> np.ndarray:
    """Y[v_full][a_full][n0] complex128 over the whole DS grid (canonical layout)."""
    nv = ds.vc.count * ds.Fv
    na = ds.ac.count * ds.Fa
    vf, af = np.meshgrid(np.arange(nv), np.arange(na), indexing="ij")
    cell, fine = ds_rows_of_canonical(ds, vf.ravel(), af.ravel())
    Y = dsgrft_rows(radar, s, ds, cell, fine, nthreads)
    return Y.reshape(nv, na, ds.r0_count)


def cfar_detect(P, cfar, K: int, nthreads: int = 0):
    """(idx int64[K'], p float64[K'], total) with K' = min(K, total)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    nv, na, nr0 = P.shape
    idx = np.zeros(max(K, 1), dtype=np.int64)
    pv = np.zeros(max(K, 1), dtype=np.float64)
    total = load().orc_cfar_detect(_p(P), nv, na, nr0, cfar.guard, cfar.train, cfar.pfa,
                                   cfar.fixed_thresh, cfar.mode, K, _p(idx), _p(pv), nthreads)
    n = min(K, int(total))
    return idx[:n], pv[:n], int(total)


def trajectory_grad(radar, s, theta, mode: int, gP=None, want_grad_s: bool = False,
                    nthreads: int = 0):
    """P[K], Y[K] complex, g[K][3] (and grad_s[M][N] complex if asked)."""
    s = _echo(s)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 3)
    K = th.shape[0]
    P = np.zeros(K)
    Y = np.zeros(K, dtype=np.complex128)
    g = np.zeros((K, 3))
    gs = np.zeros((radar.M, radar.N), dtype=np.complex128) if want_grad_s else None
    gPa = None if gP is None else np.ascontiguousarray(gP, dtype=np.float64)
    R = _radar(radar)
    load().orc_trajectory_grad(C.byref(R), _p(s), K, _p(th), mode,
                               None if gPa is None else _p(gPa), _p(P), _p(Y), _p(g),
                               None if gs is None else _p(gs), nthreads)
    return (P, Y, g, gs) if want_grad_s else (P, Y, g)


def refine(radar, s, theta, cell, steps: int, mode: int = 1, nthreads: int = 0):
    """Refined theta[K][3] and P[K]."""
    s = _echo(s)
    th = np.array(theta, dtype=np.float64).reshape(-1, 3).copy()
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    P = np.zeros(th.shape[0])
    R = _radar(radar)
    load().orc_refine(C.byref(R), _p(s), th.shape[0], _p(th), _p(cell), steps, mode, _p(P), nthreads)
    return th, P
