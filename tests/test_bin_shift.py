"""Host logic (no GPU): the range bin floor(d / dr + 1/2) of a displacement (Sec. III-A, the
bin of r(t_m) in eq. standard-GRFT-TD) as the table kernels take it (bin_shift in
csrc/internal.cuh: the quotient as a product with the rounded reciprocal, the correctly
rounded division only where the product's error could move the floor).  Checked against the
definition's IEEE operations on random displacements and on displacements within a few
units in the last place of every half-bin tie, where the bare product does pick other bins
(the test counts them, so it would catch a check that never divides).  The header is
compiled as host code by nvcc, with FMA contraction off as in the oracle."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_06788_gb300", "csrc")

PROG = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include "internal.cuh"
using namespace grft;
static uint64_t st = 0x9e3779b97f4a7c15ull;
static double uni() {                      // splitmix64 -> [0, 1)
    uint64_t z = (st += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1p-53;
}
int main() {
    const double drs[] = {15.0, 1.0, 0.3, 7.3, 0.1171875, 2.9979245800e-1, 37.5};
    long n = 0, bad = 0, product_differs = 0;
    for (double dr : drs) {
        const double inv = 1.0 / dr;
        auto check = [&](double d) {
            const int ref = (int)std::floor(d / dr + 0.5);
            const int got = bin_shift(d, dr, inv);
            const int prod = (int)std::floor(d * inv + 0.5);
            ++n;
            bad += got != ref;
            product_differs += prod != ref;
        };
        for (int i = 0; i < 2000000; ++i) check((uni() * 2.0 - 1.0) * 8000.0 * dr);
        for (int k = -4000; k <= 4000; ++k) {
            const double tie = (k + 0.5) * dr;
            double lo = tie, hi = tie;
            check(tie);
            for (int u = 0; u < 6; ++u) {
                lo = std::nextafter(lo, -INFINITY);
                hi = std::nextafter(hi, INFINITY);
                check(lo);
                check(hi);
            }
        }
    }
    printf("%ld %ld %ld\n", n, bad, product_differs);
    return 0;
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not found")


def test_bin_shift_equals_divided_bin(tmp_path):
    src = tmp_path / "bin_shift.cu"
    exe = tmp_path / "bin_shift"
    src.write_text(PROG)
    r = subprocess.run([_nvcc(), "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                        f"-I{CSRC}", str(src), "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120).stdout.split()
    n, bad, product_differs = map(int, out)
    print("checked", n, "bins; bare product differs on", product_differs)
    assert n > 14_000_000
    assert bad == 0
    assert product_differs > 0
