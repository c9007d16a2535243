"""GPU: the tile-shape autotuner of the tensor-core contraction.  Every variant (BN 256 or
128 columns, 64 or 32 k per stage with 2 to 8 stages) gives bit-identical outputs (only the
tiling differs, not the K accumulation order), with whole and ragged bin tiles; the first
call of a shape bucket records its choice in the JSON-lines cache named by
DSGRFT_TUNE_CACHE, and a later process reuses it.  The tile shapes and the tuner belong to the
4M form of the contraction (DSGRFT_PAIR=0); the pair form has one shape per product count.

The pair form (two mirrored hypotheses per contraction, the default for P = 2 grids)
matches the 4M form within the split tolerance and the FP64 oracle on every output, for
fine grids with even and odd sizes and with a fine axis of one point, in each of its tile
widths (256, 224 and 192 columns)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g, synth
from synth import Axis, DSGrid, Radar, Target
R = Radar(M=300, N=1000, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
ds = DSGrid(10, int(sys.argv[2]), Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 2), 32, 8)
s = synth.make_echo(R, [Target(400.0, -20.0, 1.0, complex(3.0, 0.0))], 9)
Y = g.dsgrft(R, torch.from_numpy(s).cuda(), ds, precision=sys.argv[3], want_Y=True, want_P=False)
assert g.grft_sync_status() == 0
np.save(sys.argv[1], Y.cpu().numpy())
"""


def _run(tmp, name, r0_count=900, precision="bf16x3", **env):
    out = os.path.join(tmp, name + ".npy")
    e = dict(os.environ)
    e.update({k: str(v) for k, v in env.items()})
    r = subprocess.run([sys.executable, "-c", CODE % ROOT, out, str(r0_count), precision], env=e, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import numpy as np
    return np.load(out)


@pytest.mark.parametrize("r0_count,precision", [(900, "bf16x3"), (800, "bf16x3"), (900, "fp16x2"), (900, "fp16x1")])
def test_tile_variants_are_bit_identical(cuda_lib, tmp_path, r0_count, precision):
    # 8 bin tiles (the last one ragged); 7; the single-product variants (twice the stages)
    import numpy as np
    y0 = _run(str(tmp_path), "v0", r0_count, precision, DSGRFT_TILE_VARIANT=0, DSGRFT_PAIR=0)
    assert np.isfinite(y0).all() and np.abs(y0).max() > 0
    for v in range(1, 3):
        yv = _run(str(tmp_path), "v%d" % v, r0_count, precision, DSGRFT_TILE_VARIANT=v, DSGRFT_PAIR=0)
        assert np.array_equal(y0, yv), v


def test_autotune_records_and_reuses_choice(cuda_lib, tmp_path):
    import numpy as np
    cache = os.path.join(str(tmp_path), "tune.jsonl")
    ya = _run(str(tmp_path), "a", DSGRFT_TUNE_CACHE=cache, DSGRFT_AUTOTUNE=1, DSGRFT_PAIR=0)
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and lines[0]["variant"] in range(3)
    assert lines[0]["Mpad"] == 320 and lines[0]["Fpad"] == 256
    yb = _run(str(tmp_path), "b", DSGRFT_TUNE_CACHE=cache, DSGRFT_AUTOTUNE=1, DSGRFT_PAIR=0)
    assert len(open(cache).readlines()) == 1          # the second process found the entry
    assert np.array_equal(ya, yb)


PAIR_CODE = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g, synth
from synth import Axis, DSGrid, Radar, Target
R = Radar(M=130, N=600, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
Fv, Fa = int(sys.argv[2]), int(sys.argv[3])
ds = DSGrid(30, 333, Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 2), Fv, Fa)
s = synth.make_echo(R, [Target(150.0, -21.0, 1.2, complex(3.0, -1.0)), Target(300.4, 3.0, -2.0, complex(1.0, 2.0))], 5)
P, Y = g.dsgrft(R, torch.from_numpy(s).cuda(), ds, precision=sys.argv[4], want_Y=True)
assert g.grft_sync_status() == 0
np.save(sys.argv[1], Y.cpu().numpy())
np.save(sys.argv[1] + ".P.npy", P.cpu().numpy())
np.save(sys.argv[1] + ".echo.npy", s)
"""


# tile widths (pair_bn): 16 x 16, 5 x 3, 7 x 1, 1 x 6 take 192 columns; 15 x 14 (119 slots) 256;
# 64 x 16 (552 slots) and 48 x 16 224; fp32: the SIMT contraction's pair form
@pytest.mark.parametrize("Fv,Fa,precision", [(16, 16, "fp16x2"), (5, 3, "fp16x2"), (7, 1, "bf16x3"), (1, 6, "fp16x1"),
                                             (64, 16, "bf16x3"), (15, 14, "fp16x2"), (48, 16, "fp16x2"),
                                             (9, 5, "fp32")])
def test_pair_form_matches_4m_form_and_oracle(cuda_lib, tmp_path, Fv, Fa, precision):
    import numpy as np
    import oracle
    from synth import Axis, DSGrid, Radar
    from tests.helpers import TOL_SPLIT, rel_peak_err

    def run(name, **env):
        out = os.path.join(str(tmp_path), name + ".npy")
        e = dict(os.environ)
        e.update({k: str(v) for k, v in env.items()})
        r = subprocess.run([sys.executable, "-c", PAIR_CODE % ROOT, out, str(Fv), str(Fa), precision], env=e,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return np.load(out), np.load(out + ".P.npy"), np.load(out + ".echo.npy")

    Yp, Pp, s = run("pair")
    Y4, P4, _ = run("m4", DSGRFT_PAIR=0)
    R = Radar(M=130, N=600, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(30, 333, Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 2), Fv, Fa)
    Yo = oracle.dsgrft_full(R, s, ds)
    ep, e4 = rel_peak_err(Yp, Yo), rel_peak_err(Y4, Yo)
    print(f"Fv={Fv} Fa={Fa} {precision}: pair form {ep:.3g}, 4M form {e4:.3g} of peak")
    assert ep <= TOL_SPLIT and e4 <= TOL_SPLIT
    assert ep <= 2 * e4 + 1e-6                        # no worse than the 4M form's rounding
    assert rel_peak_err(Yp, Y4) <= TOL_SPLIT
    assert rel_peak_err(Pp, np.abs(Yo) ** 2) <= 2 * TOL_SPLIT
