"""Host logic of the pair form (no GPU): the slot enumeration of mirrored fine hypotheses
(pair_slot / pair_slot3 in csrc/internal.cuh) lists every hypothesis of the fine grid exactly
once, pairs a hypothesis only with the one whose fine offsets are its exact negatives on
every axis (the offsets (2k - F)/2 x step/F of k and F - k; for P = 3 also the rate axis),
and leaves unpaired exactly the hypotheses with no mirror in the grid (some index 0) and the
zero-offset one; the slot count is the closed form of the enumeration.  The tile-width rule
(pair_bn) is checked against its statement on the same grids.  The header is compiled as
host code by nvcc and run here."""
import os
import shutil
import subprocess

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_06788_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <vector>
#include "internal.cuh"
using namespace grft;
int main() {
    const int grids[][3] = {{64, 16, 1}, {16, 16, 1}, {5, 3, 1}, {7, 1, 1}, {1, 6, 1}, {15, 14, 1},
                            {8, 4, 3}, {64, 8, 4}, {5, 3, 2}, {2, 2, 2}, {3, 1, 4}, {1, 5, 3}, {7, 6, 5}};
    for (auto &gr : grids) {
        const int Fv = gr[0], Fa = gr[1], Fb = gr[2], F = Fv * Fa * Fb;
        const int S = pair_slot_count3(Fv, Fa, Fb);
        std::vector<int> seen(F, 0);
        int pairs = 0, bad = 0;
        for (int s = 0; s < S; ++s) {
            int f, fm;
            pair_slot3(s, Fv, Fa, Fb, f, fm);
            if (f < 0 || f >= F) { ++bad; continue; }
            ++seen[f];
            const int u = f % Fb, k = f / Fb / Fa, q = f / Fb % Fa;
            if (fm >= 0) {
                if (fm >= F) { ++bad; continue; }
                ++seen[fm];
                ++pairs;
                const int um = fm % Fb, km = fm / Fb / Fa, qm = fm / Fb % Fa;
                // offsets negate: 2k - Fv = -(2km - Fv) on each axis (the rate axis of a P = 2
                // grid, Fb = 1, is the single zero offset)
                if (2 * k - Fv != Fv - 2 * km || 2 * q - Fa != Fa - 2 * qm) ++bad;
                if (Fb > 1 && 2 * u - Fb != Fb - 2 * um) ++bad;
            } else {
                // unpaired: an index 0 on some axis (no mirror in the grid), or the zero offset
                const bool zero = 2 * k == Fv && 2 * q == Fa && (Fb == 1 || 2 * u == Fb);
                const bool edge = k == 0 || q == 0 || (Fb > 1 && u == 0);
                if (!zero && !edge) ++bad;
            }
        }
        for (int f = 0; f < F; ++f)
            if (seen[f] != 1) ++bad;
        printf("%d %d %d %d %d %d %d\n", Fv, Fa, Fb, S, pairs, pair_bn(S), bad);
    }
    return 0;
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not found")


def test_pair_slot_enumeration_and_tile_width(tmp_path):
    src = tmp_path / "pair_slots.cu"
    exe = tmp_path / "pair_slots"
    src.write_text(PROG)
    r = subprocess.run([_nvcc(), "-std=c++17", "--expt-relaxed-constexpr", f"-I{CSRC}", str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split("\n")
    rows = [list(map(int, line.split())) for line in out if line.strip()]
    assert len(rows) == 13
    for Fv, Fa, Fb, S, pairs, bn, bad in rows:
        F = Fv * Fa * Fb
        assert bad == 0, (Fv, Fa, Fb)
        assert S == F - pairs                                  # each pair shares one slot
        if Fb == 1:
            assert S == Fa + (Fv - 1) + ((Fv - 1) * (Fa - 1) + 1) // 2
        else:
            box = (Fv - 1) * (Fa - 1) * (Fb - 1)
            assert S == Fa * Fb + (Fv - 1) * Fb + (Fv - 1) * (Fa - 1) + (box + 1) // 2
        # the tile width: fewest tiles of BN / 2 slots, then fewest columns
        cand = sorted(((-(-S // (w // 2)), -(-S // (w // 2)) * w, -w) for w in (256, 224, 192)))
        assert bn == -cand[0][2], (Fv, Fa, Fb, S, bn)
        assert bench.pair_bn(S) == bn                          # the bench's executed-FLOP factor uses it
    by_grid = {(r[0], r[1], r[2]): r for r in rows}
    assert by_grid[(64, 16, 1)][3] == 552 and by_grid[(64, 16, 1)][5] == 224
    assert by_grid[(64, 8, 4)][3] == 1387
