"""Host-side helpers of the benchmark (CPU): the residual range migration of the dual-scale
approximation on the three DS workloads (the bound holds at M=512, not at M=1024 or 2048)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


@pytest.mark.parametrize("make,residual,ok", [(synth.ds_m512, 5.12768, True),
                                              (synth.ds_adjoint_m1024, 10.91072, False),
                                              (synth.ds_precision_m2048, 24.44288, False)])
def test_residual_range_migration(make, residual, ok):
    sc = make()
    r = bench.residual_migration(sc.radar, sc.ds)
    assert r["residual_m"] == pytest.approx(residual, rel=1e-12)
    assert r["half_bin_m"] == 7.5 and r["rm_bound_ok"] is ok
