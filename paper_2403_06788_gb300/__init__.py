"""GB300 (sm_103a) GRFT / DS-GRFT coherent-sum library, after arXiv 2403.06788.

Thin PyTorch binding of libdsgrft.so (include/dsgrft.h): the functions below carry the
C ABI's names and only marshal arguments; torch provides device memory and the current
stream.  Parameter objects may be the ``synth`` dataclasses or anything with the same
attribute names (Radar: M, N, fc_hz, prf_hz, dr_m, c_mps; PlainGrid: r0_begin, r0_count,
v, a; DSGrid: r0_begin, r0_count, vc, ac, Fv, Fa; Axis: start, step, count; CFAR: guard,
train, pfa, fixed_thresh, mode).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import (DET_BYTES, GRFT_BF16X3, GRFT_FP16X1, GRFT_FP16X2, GRFT_FP16X3, GRFT_FP32, GRFT_GATHER_LINEAR,
                   GRFT_GATHER_NEAREST, PRECISIONS, GrftError, check, load)

__all__ = ["dsgrft3_fine_dfm", "dsgrft3", "dsgrft_coarse_rm_fd_ex", "dsgrft_fine_dfm_fd", "dsgrft_fd", "dskt_keystone", "spectral_slots", "dskt_coarse_rm", "dskt_fine_dfm_fft", "dskt_mfp", "dsktmfp",
           "load", "grft_version", "grft_sync_status", "grft_set_wait_limit", "grft_release_workspace",
           "grft_shutdown",
           "grft_selftest_wait", "grft_timing", "grft_timing_get",
           "grft_bins_phases", "grft_plain", "grft_plain_static", "dsgrft_coarse_rm", "dsgrft_fine_dfm",
           "dsgrft_fine_dfm_batched", "dsgrft_fine_dfm_fft", "dsgrft_coarse_rm_fd", "detect_peaks", "dsgrft_backward", "dsgrft_refine",
           "detect_peaks_begin", "detect_peaks_add", "detect_peaks_end", "detect_merge", "dsgrft_detect",
           "grft", "dsgrft", "decode_detections", "TrajectoryPower", "GrftError",
           "GRFT_FP32", "GRFT_BF16X3", "GRFT_FP16X3", "GRFT_FP16X1", "GRFT_FP16X2", "GRFT_GATHER_NEAREST", "GRFT_GATHER_LINEAR"]

DET_DTYPE = np.dtype([("idx", "<i8"), ("n0", "<i4"), ("vi", "<i4"), ("ai", "<i4"), ("p", "<f4"),
                      ("r0_m", "<f8"), ("v", "<f8"), ("a", "<f8")])
assert DET_DTYPE.itemsize == DET_BYTES


# ----------------------------------------------------------------------------- marshalling
def _axis(a) -> _abi.grft_axis:
    return _abi.grft_axis(float(a.start), float(a.step), int(a.count), 0)


def _radar(r) -> _abi.grft_radar:
    return _abi.grft_radar(int(r.M), int(r.N), float(r.fc_hz), float(r.prf_hz), float(r.dr_m),
                           float(getattr(r, "c_mps", 3.0e8)))


def _grid(g) -> _abi.grft_grid:
    return _abi.grft_grid(int(g.r0_begin), int(g.r0_count), _axis(g.v), _axis(g.a))


def _dsgrid(g) -> _abi.grft_dsgrid:
    return _abi.grft_dsgrid(int(g.r0_begin), int(g.r0_count), _axis(g.vc), _axis(g.ac), int(g.Fv),
                            int(g.Fa))


def _dsgrid3(g) -> _abi.grft_dsgrid3:
    return _abi.grft_dsgrid3(int(g.r0_begin), int(g.r0_count), _axis(g.vc), _axis(g.ac), _axis(g.bc), int(g.Fv),
                             int(g.Fa), int(g.Fb))


def _cfar(c) -> _abi.grft_cfar:
    return _abi.grft_cfar(int(c.guard), int(c.train), float(c.pfa), float(c.fixed_thresh), int(c.mode))


def _precision(p) -> int:
    if isinstance(p, str):
        return PRECISIONS[p.lower()]
    return int(p)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- C ABI names
def grft_version() -> int:
    return int(load().grft_version())


def grft_sync_status(stream=None) -> int:
    return int(load().grft_sync_status(_stream(stream)))


def grft_set_wait_limit(cycles: int) -> None:
    check(load().grft_set_wait_limit(int(cycles)), "grft_set_wait_limit")


def grft_release_workspace() -> None:
    check(load().grft_release_workspace(), "grft_release_workspace")


def grft_shutdown() -> None:
    """Release the current device's workspaces, pipeline stream/events and timing events."""
    check(load().grft_shutdown(), "grft_shutdown")


def grft_timing(enable: bool) -> None:
    """Per-kernel CUDA-event timing on (clears the totals) or off."""
    check(load().grft_timing(1 if enable else 0), "grft_timing")


def grft_timing_get(kernel):
    """(launches, total_ms) of a kernel class ('contract', 'split', 'cfar', ...); synchronises."""
    k = _abi.KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    n, ms = C.c_int32(0), C.c_double(0.0)
    check(load().grft_timing_get(k, C.byref(n), C.byref(ms)), "grft_timing_get")
    return int(n.value), float(ms.value)


def grft_selftest_wait(cycles: int, stream=None) -> None:
    check(load().grft_selftest_wait(int(cycles), _stream(stream)), "grft_selftest_wait")


def grft_bins_phases(radar, v, a, rho, w, stream=None):
    nh = int(v.numel())
    R = _radar(radar)
    check(load().grft_bins_phases(C.byref(R), _ptr(v, torch.float64, "v"), _ptr(a, torch.float64, "a"),
                                  nh, _ptr(rho, torch.int32, "rho"), _ptr(w, torch.complex64, "w"),
                                  _stream(stream)), "grft_bins_phases")


def grft_plain(radar, echo, grid, Y=None, P=None, stream=None):
    R, G = _radar(radar), _grid(grid)
    check(load().grft_plain(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                            _ptr(Y, torch.complex64, "Y"), _ptr(P, torch.float32, "P"),
                            _stream(stream)), "grft_plain")


def grft_plain_static(radar, echo, grid, Y=None, P=None, stream=None):
    """grft_plain without any device allocation (fixed in-library scratch; see the header)."""
    R, G = _radar(radar), _grid(grid)
    check(load().grft_plain_static(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                                   _ptr(Y, torch.complex64, "Y"), _ptr(P, torch.float32, "P"),
                                   _stream(stream)), "grft_plain_static")


def dsgrft_coarse_rm(radar, echo, grid, cell_begin, cell_count, Z, stream=None):
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_coarse_rm(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                                  int(cell_begin), int(cell_count), _ptr(Z, torch.complex64, "Z"),
                                  _stream(stream)), "dsgrft_coarse_rm")


def dsgrft_fine_dfm(radar, Z, echo, grid, cell_begin, cell_count, precision, Y=None, P=None,
                    stream=None):
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_fine_dfm(C.byref(R), _ptr(Z, torch.complex64, "Z"),
                                 _ptr(echo, torch.complex64, "echo"), C.byref(G), int(cell_begin),
                                 int(cell_count), _precision(precision), _ptr(Y, torch.complex64, "Y"),
                                 _ptr(P, torch.float32, "P"), _stream(stream)), "dsgrft_fine_dfm")


def dsgrft_coarse_rm_fd(radar, echo, grid, cell_begin, cell_count, Z, stream=None):
    """Frequency-domain coarse stage (mGIFT, Alg. 1) into Z [cell_count][M][r0_count]."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_coarse_rm_fd(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                                     int(cell_begin), int(cell_count), _ptr(Z, torch.complex64, "Z"),
                                     _stream(stream)), "dsgrft_coarse_rm_fd")


def dsgrft_coarse_rm_fd_ex(radar, echo, grid, cell_begin, cell_count, band, Z, stream=None):
    """Frequency-domain coarse stage over `band` ('baseband' or 'positive', the paper's
    discrete band k = 0..N-1) into Z [cell_count][M][r0_count]."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_coarse_rm_fd_ex(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                                        int(cell_begin), int(cell_count), _abi.BANDS[band],
                                        _ptr(Z, torch.complex64, "Z"), _stream(stream)), "dsgrft_coarse_rm_fd_ex")


def dsgrft_fine_dfm_fd(radar, Z, grid, cell_begin, cell_count, band, precision, Y=None, P=None, stream=None):
    """Fine stage on Z of dsgrft_coarse_rm_fd_ex with the same band (fine offsets scaled for
    the positive band, Prop. 1)."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_fine_dfm_fd(C.byref(R), _ptr(Z, torch.complex64, "Z"), C.byref(G), int(cell_begin),
                                    int(cell_count), _abi.BANDS[band], _precision(precision),
                                    _ptr(Y, torch.complex64, "Y"), _ptr(P, torch.float32, "P"), _stream(stream)),
          "dsgrft_fine_dfm_fd")


def dsgrft_fd(radar, echo, grid, band="baseband", precision="bf16x3", want_Y=False, want_P=True):
    """DS-GRFT with the frequency-domain coarse stage (the paper's form, Alg. 1 + Alg. 3) over
    the whole grid; returns P [v_full][a_full][r0] (and Y)."""
    nv, na = int(grid.vc.count) * int(grid.Fv), int(grid.ac.count) * int(grid.Fa)
    shape = (nv, na, int(grid.r0_count))
    P = torch.empty(shape, dtype=torch.float32, device=echo.device) if want_P else None
    Y = torch.empty(shape, dtype=torch.complex64, device=echo.device) if want_Y else None
    ncell = int(grid.vc.count) * int(grid.ac.count)
    Z = torch.empty((ncell, int(echo.shape[0]), int(grid.r0_count)), dtype=torch.complex64, device=echo.device)
    dsgrft_coarse_rm_fd_ex(radar, echo, grid, 0, ncell, band, Z)
    dsgrft_fine_dfm_fd(radar, Z, grid, 0, ncell, band, precision, Y, P)
    if want_Y and want_P:
        return P, Y
    return Y if want_Y else P


def dsgrft_fine_dfm_fft(radar, echo, grid, cell_begin, cell_count, Y=None, P=None, stream=None):
    """FFT form of the fine stage (Alg. 2); the grid's fine velocity step must be one Doppler
    bin of a 256- or 512-point transform (else GrftError with GRFT_EUNSUPPORTED)."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dsgrft_fine_dfm_fft(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                                     int(cell_begin), int(cell_count), _ptr(Y, torch.complex64, "Y"),
                                     _ptr(P, torch.float32, "P"), _stream(stream)), "dsgrft_fine_dfm_fft")


def dsgrft3_fine_dfm(radar, echo, grid3, cell_begin, cell_count, precision, Y=None, P=None, stream=None):
    """DS-GRFT with the acceleration rate (P = 3), fused gather + tensor-core contraction into
    the v-slab [(i - i0) Fv + k][l Fa + q][w Fb + u][r0] starting at i0 = cell_begin / (na nb)."""
    R, G = _radar(radar), _dsgrid3(grid3)
    check(load().dsgrft3_fine_dfm(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G), int(cell_begin),
                                  int(cell_count), _precision(precision), _ptr(Y, torch.complex64, "Y"),
                                  _ptr(P, torch.float32, "P"), _stream(stream)), "dsgrft3_fine_dfm")


def dsgrft3(radar, echo, grid3, precision="bf16x3", want_Y=False, want_P=True):
    """P = 3 DS-GRFT over the whole grid; returns P [v_full][a_full][b_full][r0] (and Y)."""
    shape = (int(grid3.vc.count) * int(grid3.Fv), int(grid3.ac.count) * int(grid3.Fa),
             int(grid3.bc.count) * int(grid3.Fb), int(grid3.r0_count))
    P = torch.empty(shape, dtype=torch.float32, device=echo.device) if want_P else None
    Y = torch.empty(shape, dtype=torch.complex64, device=echo.device) if want_Y else None
    ncell = int(grid3.vc.count) * int(grid3.ac.count) * int(grid3.bc.count)
    dsgrft3_fine_dfm(radar, echo, grid3, 0, ncell, precision, Y, P)
    if want_Y and want_P:
        return P, Y
    return Y if want_Y else P


def dskt_keystone(radar, echo, Skt, stream=None):
    """Range spectra and keystone transform (eq. Echo-after-KT) into Skt [M][N]; range-
    frequency slot p holds frequency index bitrev(p) (see spectral_slots)."""
    R = _radar(radar)
    check(load().dskt_keystone(C.byref(R), _ptr(echo, torch.complex64, "echo"), _ptr(Skt, torch.complex64, "Skt"),
                               _stream(stream)), "dskt_keystone")


def spectral_slots(N: int):
    """Frequency index (FFT order, 0..N-1) held by each range-frequency slot of Skt: the
    bit reversal of the slot over log2(N) bits (host list)."""
    bits = int(N).bit_length() - 1
    return [int(format(p, f"0{bits}b")[::-1], 2) if bits else 0 for p in range(int(N))]


def dskt_coarse_rm(radar, Skt, grid, cell_begin, cell_count, Z, stream=None):
    """Coarse stage of DS-KT-MFP (Cor. 1: H_KT,RM and H_pre-DFM) into Z [cell_count][M][r0_count]."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dskt_coarse_rm(C.byref(R), _ptr(Skt, torch.complex64, "Skt"), C.byref(G), int(cell_begin),
                                int(cell_count), _ptr(Z, torch.complex64, "Z"), _stream(stream)), "dskt_coarse_rm")


def dskt_fine_dfm_fft(radar, Z, grid, cell_begin, cell_count, Y=None, P=None, stream=None):
    """Fine stage of DS-KT-MFP (Prop. 3, FFT form of the GFT) on Z of dskt_coarse_rm."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dskt_fine_dfm_fft(C.byref(R), _ptr(Z, torch.complex64, "Z"), C.byref(G), int(cell_begin),
                                   int(cell_count), _ptr(Y, torch.complex64, "Y"), _ptr(P, torch.float32, "P"),
                                   _stream(stream)), "dskt_fine_dfm_fft")


def dskt_mfp(radar, echo, grid, Y=None, P=None, stream=None):
    """The whole DS-KT-MFP map (Alg. 4) into Y and/or P [nq Fv][nac Fa][r0_count]."""
    R, G = _radar(radar), _dsgrid(grid)
    check(load().dskt_mfp(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G),
                          _ptr(Y, torch.complex64, "Y"), _ptr(P, torch.float32, "P"), _stream(stream)), "dskt_mfp")


def dsktmfp(radar, echo, grid, want_Y=False, want_P=True):
    """DS-KT-MFP over the whole keystone grid; returns P [v_full][a_full][r0] (and Y)."""
    nv, na = int(grid.vc.count) * int(grid.Fv), int(grid.ac.count) * int(grid.Fa)
    shape = (nv, na, int(grid.r0_count))
    P = torch.empty(shape, dtype=torch.float32, device=echo.device) if want_P else None
    Y = torch.empty(shape, dtype=torch.complex64, device=echo.device) if want_Y else None
    dskt_mfp(radar, echo, grid, Y, P)
    if want_Y and want_P:
        return P, Y
    return Y if want_Y else P


def dsgrft_fine_dfm_batched(radar, grid, items, precision, stream=None):
    """items: list of dicts with keys echo (complex64 [M][N]), P, Y (either may be None),
    r0_begin, r0_count."""
    R, G = _radar(radar), _dsgrid(grid)
    arr = (_abi.grft_batch_item * len(items))()
    for i, it in enumerate(items):
        e = it["echo"]
        arr[i].echo = _ptr(e, torch.complex64, "echo").value
        arr[i].P = _ptr(it.get("P"), torch.float32, "P").value if it.get("P") is not None else None
        arr[i].Y = _ptr(it.get("Y"), torch.complex64, "Y").value if it.get("Y") is not None else None
        arr[i].M, arr[i].N = int(e.shape[0]), int(e.shape[1])
        arr[i].r0_begin = int(it.get("r0_begin", 0))
        arr[i].r0_count = int(it.get("r0_count", e.shape[1]))
    check(load().dsgrft_fine_dfm_batched(C.byref(R), C.byref(G), arr, len(items), _precision(precision),
                                         _stream(stream)), "dsgrft_fine_dfm_batched")


def detect_peaks(P, cfar, K, axes=None, dr_m=0.0, out=None, n_out=None, stream=None):
    """P: float32 [nv][na][nr0] CUDA tensor.  Returns (out, n_out) device tensors: out is a
    uint8 buffer of K grft_det records, n_out an int32 scalar (total detections)."""
    if P.dim() != 3:
        raise ValueError("P must be [nv][na][nr0]")
    nv, na, nr0 = (int(x) for x in P.shape)
    if out is None:
        out = torch.zeros(max(int(K), 1) * DET_BYTES, dtype=torch.uint8, device=P.device)
    if n_out is None:
        n_out = torch.zeros(1, dtype=torch.int32, device=P.device)
    Cf = _cfar(cfar)
    A = _grid(axes) if axes is not None else None
    check(load().detect_peaks(_ptr(P, torch.float32, "P"), nv, na, nr0, C.byref(Cf),
                              C.byref(A) if A is not None else None, float(dr_m), int(K),
                              _ptr(out, torch.uint8, "out"), _ptr(n_out, torch.int32, "n_out"),
                              _stream(stream)), "detect_peaks")
    return out, n_out


def _det_buffers(K, device, out, n_out):
    if out is None:
        out = torch.zeros(max(int(K), 1) * DET_BYTES, dtype=torch.uint8, device=device)
    if n_out is None:
        n_out = torch.zeros(1, dtype=torch.int32, device=device)
    return out, n_out


def detect_peaks_begin(stream=None):
    check(load().detect_peaks_begin(_stream(stream)), "detect_peaks_begin")


def detect_peaks_add(P, v_lo, v_hi, v_base, cfar, stream=None):
    """Scan slab P [nv][na][nr0] (rows v_base + r of the whole map); rows outside [v_lo, v_hi)
    are the halo (neighbours only)."""
    if P.dim() != 3:
        raise ValueError("P must be [nv][na][nr0]")
    nv, na, nr0 = (int(x) for x in P.shape)
    Cf = _cfar(cfar)
    check(load().detect_peaks_add(_ptr(P, torch.float32, "P"), nv, na, nr0, int(v_lo), int(v_hi), int(v_base),
                                  C.byref(Cf), _stream(stream)), "detect_peaks_add")


def detect_peaks_end(na, nr0, K, axes=None, dr_m=0.0, out=None, n_out=None, device="cuda", stream=None):
    out, n_out = _det_buffers(K, device, out, n_out)
    A = _grid(axes) if axes is not None else None
    check(load().detect_peaks_end(int(na), int(nr0), C.byref(A) if A is not None else None, float(dr_m), int(K),
                                  _ptr(out, torch.uint8, "out"), _ptr(n_out, torch.int32, "n_out"),
                                  _stream(stream)), "detect_peaks_end")
    return out, n_out


def detect_merge(lists, totals, K_in, K, out=None, n_out=None, stream=None):
    """lists: uint8 CUDA buffer of n_lists * K_in grft_det records; totals: int32 CUDA tensor
    [n_lists].  Returns (out, n_out): the top K of the union (see the header)."""
    n_lists = int(totals.numel())
    out, n_out = _det_buffers(K, totals.device, out, n_out)
    check(load().detect_merge(_ptr(lists, torch.uint8, "lists"), _ptr(totals, torch.int32, "totals"), n_lists,
                              int(K_in), int(K), _ptr(out, torch.uint8, "out"), _ptr(n_out, torch.int32, "n_out"),
                              _stream(stream)), "detect_merge")
    return out, n_out


def dsgrft_detect(radar, echo, grid, precision, cfar, K, out=None, n_out=None, stream=None):
    """DS-GRFT over the whole dual-scale grid with streamed detection (the power map is never
    held whole).  Returns (out, n_out) as detect_peaks."""
    out, n_out = _det_buffers(K, echo.device, out, n_out)
    R, G, Cf = _radar(radar), _dsgrid(grid), _cfar(cfar)
    check(load().dsgrft_detect(C.byref(R), _ptr(echo, torch.complex64, "echo"), C.byref(G), _precision(precision),
                               C.byref(Cf), int(K), _ptr(out, torch.uint8, "out"), _ptr(n_out, torch.int32, "n_out"),
                               _stream(stream)), "dsgrft_detect")
    return out, n_out


def decode_detections(out, n_out, K):
    """Host copy of the detections as a numpy structured array (synchronises)."""
    total = int(n_out.item())
    n = min(total, int(K))
    raw = out[: n * DET_BYTES].cpu().numpy()
    return np.frombuffer(raw.tobytes(), dtype=DET_DTYPE, count=n), total


def dsgrft_backward(radar, echo, theta, gather, grad_P=None, P=None, Y=None, grad_theta=None,
                    grad_s=None, stream=None):
    R = _radar(radar)
    K = int(theta.shape[0])
    check(load().dsgrft_backward(C.byref(R), _ptr(echo, torch.complex64, "echo"), K,
                                 _ptr(theta, torch.float64, "theta"), int(gather),
                                 _ptr(grad_P, torch.float32, "grad_P"), _ptr(P, torch.float32, "P"),
                                 _ptr(Y, torch.complex64, "Y"),
                                 _ptr(grad_theta, torch.float64, "grad_theta"),
                                 _ptr(grad_s, torch.complex64, "grad_s"), _stream(stream)),
          "dsgrft_backward")


def dsgrft_refine(radar, echo, theta, cell, steps, gather, P_out, stream=None):
    R = _radar(radar)
    cell_arr = (C.c_double * 3)(*[float(x) for x in cell])
    check(load().dsgrft_refine(C.byref(R), _ptr(echo, torch.complex64, "echo"), int(theta.shape[0]),
                               _ptr(theta, torch.float64, "theta"), cell_arr, int(steps), int(gather),
                               _ptr(P_out, torch.float32, "P_out"), _stream(stream)), "dsgrft_refine")


# ----------------------------------------------------------------------------- conveniences
def grft(radar, echo, grid, want_Y=False):
    """Plain GRFT over the whole grid; returns P [v][a][r0] (and Y if asked)."""
    shape = (int(grid.v.count), int(grid.a.count), int(grid.r0_count))
    P = torch.empty(shape, dtype=torch.float32, device=echo.device)
    Y = torch.empty(shape, dtype=torch.complex64, device=echo.device) if want_Y else None
    grft_plain(radar, echo, grid, Y, P)
    return (P, Y) if want_Y else P


def dsgrft(radar, echo, grid, precision="bf16x3", want_Y=False, want_P=True, fused=True):
    """DS-GRFT over the whole dual-scale grid; returns P [v_full][a_full][r0] (and Y)."""
    nv, na = int(grid.vc.count) * int(grid.Fv), int(grid.ac.count) * int(grid.Fa)
    shape = (nv, na, int(grid.r0_count))
    P = torch.empty(shape, dtype=torch.float32, device=echo.device) if want_P else None
    Y = torch.empty(shape, dtype=torch.complex64, device=echo.device) if want_Y else None
    ncell = int(grid.vc.count) * int(grid.ac.count)
    Z = None
    if not fused:
        Z = torch.empty((ncell, int(echo.shape[0]), int(grid.r0_count)), dtype=torch.complex64,
                        device=echo.device)
        dsgrft_coarse_rm(radar, echo, grid, 0, ncell, Z)
    dsgrft_fine_dfm(radar, Z, echo, grid, 0, ncell, precision, Y, P)
    if want_Y and want_P:
        return P, Y
    return Y if want_Y else P


class TrajectoryPower(torch.autograd.Function):
    """P_k = |Y(theta_k)|^2 along continuous trajectories theta [K][3] = (r0_m, v, a), with the
    hand-written adjoint for d/d theta and d/d echo (linear gather by default)."""

    @staticmethod
    def forward(ctx, echo, theta, radar, gather=GRFT_GATHER_LINEAR):
        K = theta.shape[0]
        P = torch.empty(K, dtype=torch.float32, device=echo.device)
        th = theta.detach().contiguous()
        dsgrft_backward(radar, echo.detach().contiguous(), th, gather, P=P)
        ctx.save_for_backward(echo, th)
        ctx.radar, ctx.gather = radar, gather
        return P

    @staticmethod
    def backward(ctx, gP):
        echo, th = ctx.saved_tensors
        gP = gP.detach().to(torch.float32).contiguous()
        g_th = torch.zeros_like(th) if ctx.needs_input_grad[1] else None
        g_s = torch.zeros_like(echo) if ctx.needs_input_grad[0] else None
        dsgrft_backward(ctx.radar, echo.detach().contiguous(), th, ctx.gather, grad_P=gP,
                        grad_theta=g_th, grad_s=g_s)
        return g_s, g_th, None, None
