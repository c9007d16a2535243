"""GPU: the tile shapes of the plain GRFT kernel (eq. standard-GRFT-TD), 8 x 4 (the default),
8 x 2 and 16 x 2 hypotheses x bins per thread (DSGRFT_PLAIN_SHAPE), give the same results bit for bit and match
the FP64 oracle on every output within the FP32 tolerance.  The grid mixes hypotheses whose
bin shifts differ inside a CTA's group (the per-hypothesis reload path) with ones that share
it, over a ragged pulse count, a partial last group and bins that leave the echo at both
edges."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from synth import Axis, PlainGrid, Radar, Target
from tests.helpers import TOL_FP32, rel_peak_err

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # accelerations 40 m/s^2 apart at 1 m bins: shifts differ inside a group of 8 hypotheses
    "mixed": (Radar(M=300, N=1200, fc_hz=1.5e9, prf_hz=1000.0, dr_m=1.0),
              PlainGrid(3, 1190, Axis(-30.0, 7.5, 5), Axis(-200.0, 40.0, 11))),
    # the usual case: neighbouring accelerations share the shift at (almost) every pulse
    "shared": (Radar(M=133, N=2100, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0),
               PlainGrid(0, 2100, Axis(-280.0, 61.3, 6), Axis(-18.0, 4.4, 9))),
}

CODE = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g, synth
from tests.test_gpu_plain_shapes import CASES, echo_of
R, grid = CASES[sys.argv[2]]
s = echo_of(R)
P, Y = g.grft(R, torch.from_numpy(s).cuda(), grid, want_Y=True)
assert g.grft_sync_status() == 0
np.save(sys.argv[1], Y.cpu().numpy())
"""


def echo_of(R):
    return synth.make_echo(R, [Target(R.N / 2, -15.0, -3.0, complex(2.0, 1.0)),
                               Target(R.N / 5, -7.5, 10.0, complex(0.0, 3.0))], 11)


def _run(tmp, case, shape):
    out = os.path.join(tmp, "%s_%s.npy" % (case, shape))
    e = dict(os.environ)
    e["DSGRFT_PLAIN_SHAPE"] = shape
    r = subprocess.run([sys.executable, "-c", CODE % ROOT, out, case], env=e, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


@pytest.mark.parametrize("case", sorted(CASES))
def test_plain_shapes_match_oracle_and_agree(cuda_lib, tmp_path, case):
    R, grid = CASES[case]
    Yo = oracle.grft_plain_full(R, echo_of(R), grid)
    Ys = {shape: _run(str(tmp_path), case, shape) for shape in ("8x2", "8x4", "16x2")}
    for shape, Y in Ys.items():
        err = rel_peak_err(Y, Yo)
        print(case, shape, "max rel peak err", err)
        assert err <= TOL_FP32, shape
    assert np.array_equal(Ys["8x2"], Ys["8x4"]) and np.array_equal(Ys["8x2"], Ys["16x2"])
