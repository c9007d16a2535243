"""ctypes binding of libdsgrft.so (include/dsgrft.h).  Argument marshalling only: every
step of the path runs in the library's CUDA kernels.  There is no CPU fallback; a
missing or unloadable library raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

GRFT_OK, GRFT_EINVAL, GRFT_ENOMEM, GRFT_ECUDA, GRFT_ETIMEOUT, GRFT_EUNSUPPORTED, GRFT_EOVERFLOW = (
    0, -1, -2, -3, -4, -5, -6)
GRFT_FP32, GRFT_BF16X3, GRFT_FP16X3, GRFT_FP16X1, GRFT_FP16X2 = 0, 1, 2, 3, 4
GRFT_GATHER_NEAREST, GRFT_GATHER_LINEAR = 0, 1
BANDS = {"baseband": 0, "positive": 1}
PRECISIONS = {"fp32": GRFT_FP32, "bf16x3": GRFT_BF16X3, "fp16x3": GRFT_FP16X3, "fp16x1": GRFT_FP16X1,
              "fp16x2": GRFT_FP16X2}
KERNELS = {"tables": 0, "plain": 1, "coarse_rm": 2, "split": 3, "contract": 4, "contract_fp32": 5,
           "cfar": 6, "topk": 7, "adjoint": 8, "contract_fft": 9, "keystone": 10}


class grft_axis(C.Structure):
    _fields_ = [("start", C.c_double), ("step", C.c_double), ("count", C.c_int32),
                ("reserved", C.c_int32)]


class grft_radar(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("fc_hz", C.c_double), ("prf_hz", C.c_double),
                ("dr_m", C.c_double), ("c_mps", C.c_double)]


class grft_grid(C.Structure):
    _fields_ = [("r0_begin", C.c_int32), ("r0_count", C.c_int32), ("v", grft_axis), ("a", grft_axis)]


class grft_dsgrid(C.Structure):
    _fields_ = [("r0_begin", C.c_int32), ("r0_count", C.c_int32), ("vc", grft_axis),
                ("ac", grft_axis), ("Fv", C.c_int32), ("Fa", C.c_int32)]


class grft_dsgrid3(C.Structure):
    _fields_ = [("r0_begin", C.c_int32), ("r0_count", C.c_int32), ("vc", grft_axis),
                ("ac", grft_axis), ("bc", grft_axis), ("Fv", C.c_int32), ("Fa", C.c_int32), ("Fb", C.c_int32)]


class grft_cfar(C.Structure):
    _fields_ = [("guard", C.c_int32), ("train", C.c_int32), ("pfa", C.c_double),
                ("fixed_thresh", C.c_float), ("mode", C.c_int32)]


class grft_det(C.Structure):
    _fields_ = [("idx", C.c_int64), ("n0", C.c_int32), ("vi", C.c_int32), ("ai", C.c_int32),
                ("p", C.c_float), ("r0_m", C.c_double), ("v", C.c_double), ("a", C.c_double)]


class grft_batch_item(C.Structure):
    _fields_ = [("echo", C.c_void_p), ("P", C.c_void_p), ("Y", C.c_void_p), ("M", C.c_int32),
                ("N", C.c_int32), ("r0_begin", C.c_int32), ("r0_count", C.c_int32)]


DET_BYTES = C.sizeof(grft_det)

# symbol -> (restype, argtypes); the list every test checks against include/dsgrft.h
_P = C.c_void_p
SIGNATURES = {
    "grft_version": (C.c_int, []),
    "grft_status_string": (C.c_char_p, [C.c_int]),
    "grft_sync_status": (C.c_int, [_P]),
    "grft_set_wait_limit": (C.c_int, [C.c_uint64]),
    "grft_release_workspace": (C.c_int, []),
    "grft_shutdown": (C.c_int, []),
    "grft_selftest_wait": (C.c_int, [C.c_uint64, _P]),
    "grft_timing": (C.c_int, [C.c_int]),
    "grft_timing_get": (C.c_int, [C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "grft_bins_phases": (C.c_int, [C.POINTER(grft_radar), _P, _P, C.c_int32, _P, _P, _P]),
    "grft_plain": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_grid), _P, _P, _P]),
    "grft_plain_static": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_grid), _P, _P, _P]),
    "dsgrft_coarse_rm": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32,
                                   C.c_int32, _P, _P]),
    "dsgrft_fine_dfm": (C.c_int, [C.POINTER(grft_radar), _P, _P, C.POINTER(grft_dsgrid), C.c_int32,
                                  C.c_int32, C.c_int, _P, _P, _P]),
    "dsgrft_coarse_rm_fd": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32,
                                      C.c_int32, _P, _P]),
    "dsgrft_coarse_rm_fd_ex": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32, C.c_int32,
                                         C.c_int, _P, _P]),
    "dsgrft_fine_dfm_fd": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32, C.c_int32,
                                     C.c_int, C.c_int, _P, _P, _P]),
    "dsgrft_fine_dfm_fft": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32,
                                      C.c_int32, _P, _P, _P]),
    "dsgrft3_fine_dfm": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid3), C.c_int32, C.c_int32,
                                   C.c_int, _P, _P, _P]),
    "dskt_keystone": (C.c_int, [C.POINTER(grft_radar), _P, _P, _P]),
    "dskt_coarse_rm": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32, C.c_int32, _P, _P]),
    "dskt_fine_dfm_fft": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int32, C.c_int32,
                                    _P, _P, _P]),
    "dskt_mfp": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), _P, _P, _P]),
    "dsgrft_fine_dfm_batched": (C.c_int, [C.POINTER(grft_radar), C.POINTER(grft_dsgrid),
                                          C.POINTER(grft_batch_item), C.c_int32, C.c_int, _P]),
    "detect_peaks": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(grft_cfar),
                               C.POINTER(grft_grid), C.c_double, C.c_int32, _P, _P, _P]),
    "detect_peaks_begin": (C.c_int, [_P]),
    "detect_peaks_add": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                   C.POINTER(grft_cfar), _P]),
    "detect_peaks_end": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(grft_grid), C.c_double, C.c_int32, _P, _P,
                                   _P]),
    "detect_merge": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]),
    "dsgrft_detect": (C.c_int, [C.POINTER(grft_radar), _P, C.POINTER(grft_dsgrid), C.c_int, C.POINTER(grft_cfar),
                                C.c_int32, _P, _P, _P]),
    "dsgrft_backward": (C.c_int, [C.POINTER(grft_radar), _P, C.c_int32, _P, C.c_int, _P, _P, _P, _P,
                                  _P, _P]),
    "dsgrft_refine": (C.c_int, [C.POINTER(grft_radar), _P, C.c_int32, _P, C.POINTER(C.c_double),
                                C.c_int32, C.c_int, _P, _P]),
}


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libdsgrft.so")


def load(build_if_missing: bool = True):
    """Load (building first if needed) libdsgrft.so and declare every exported signature."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if build_if_missing:
            from .build import build
            path = build()
        if not os.path.exists(path):
            raise RuntimeError(f"libdsgrft.so is not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GrftError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().grft_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != GRFT_OK:
        raise GrftError(code, where)
