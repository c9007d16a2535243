"""The C-ABI library builds, loads and exports every symbol include/dsgrft.h declares
(no compute calls: CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsgrft.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("grft_plain", "dsgrft_coarse_rm", "dsgrft_fine_dfm", "detect_peaks", "dsgrft_backward",
              "dsgrft_refine", "dsgrft_fine_dfm_batched", "grft_bins_phases"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2403_06788_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)          # loads without a GPU (CUDA runtime is linked statically)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (\w+)$", out, flags=re.M))
    assert set(_declared()) <= exported


def test_binding_declares_signatures_for_every_symbol():
    from paper_2403_06788_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(_declared())


def test_struct_layouts_match_header_sizes():
    from paper_2403_06788_gb300 import _abi
    assert ctypes.sizeof(_abi.grft_axis) == 24
    assert ctypes.sizeof(_abi.grft_radar) == 40
    assert ctypes.sizeof(_abi.grft_grid) == 56
    assert ctypes.sizeof(_abi.grft_dsgrid) == 64
    assert ctypes.sizeof(_abi.grft_det) == 48
    assert ctypes.sizeof(_abi.grft_cfar) == 24


def test_struct_offsets_compiled_by_the_host_compiler():
    """Compile a probe against the header with gcc and compare offsets with ctypes."""
    import tempfile
    from paper_2403_06788_gb300 import _abi
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "dsgrft.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(grft_det), offsetof(grft_det,p), offsetof(grft_det,r0_m),
   sizeof(grft_dsgrid), offsetof(grft_dsgrid,Fv), sizeof(grft_batch_item), offsetof(grft_cfar,fixed_thresh),
   sizeof(grft_dsgrid3), offsetof(grft_dsgrid3,bc), offsetof(grft_dsgrid3,Fb));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(_abi.grft_det), _abi.grft_det.p.offset, _abi.grft_det.r0_m.offset,
                    ctypes.sizeof(_abi.grft_dsgrid), _abi.grft_dsgrid.Fv.offset,
                    ctypes.sizeof(_abi.grft_batch_item), _abi.grft_cfar.fixed_thresh.offset,
                    ctypes.sizeof(_abi.grft_dsgrid3), _abi.grft_dsgrid3.bc.offset, _abi.grft_dsgrid3.Fb.offset]


def test_kernel_class_ids_match_header():
    """The binding's kernel-class names carry the values of the header's GRFT_KERNEL_* enum."""
    import re
    from paper_2403_06788_gb300 import _abi
    text = open(HEADER).read()
    enum = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"GRFT_KERNEL_([A-Z0-9_]+)\s*=\s*(\d+)", text)}
    count = enum.pop("count")
    assert enum == _abi.KERNELS
    assert count == len(enum) == max(enum.values()) + 1
