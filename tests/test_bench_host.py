"""Host-side helpers of the benchmark (CPU): the residual range migration of the dual-scale
approximation on the three DS workloads (the bound holds at M=512, not at M=1024 or 2048),
and the oracle's per-call thread count that the CPU baseline relies on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


@pytest.mark.parametrize("make,residual,ok", [(synth.ds_m512, 5.12768, True),
                                              (synth.ds_adjoint_m1024, 10.91072, False),
                                              (synth.ds_precision_m2048, 24.44288, False)])
def test_residual_range_migration(make, residual, ok):
    sc = make()
    r = bench.residual_migration(sc.radar, sc.ds)
    assert r["residual_m"] == pytest.approx(residual, rel=1e-12)
    assert r["half_bin_m"] == 7.5 and r["rm_bound_ok"] is ok


def test_oracle_thread_count_of_a_call_does_not_persist():
    """A one-thread call gives the same rows as an all-thread call and leaves the default
    thread count of later calls unchanged (the CPU baseline times both in one process)."""
    sc = synth.ds_m512()
    s = synth.make_echo(sc.radar, sc.targets, sc.seed)
    cells, fine = np.arange(4) * 37, np.arange(4) * 101
    default = oracle.num_threads()
    Ya = oracle.dsgrft_rows(sc.radar, s, sc.ds, cells, fine)
    Y1 = oracle.dsgrft_rows(sc.radar, s, sc.ds, cells, fine, nthreads=1)
    assert oracle.num_threads() == default
    Yb = oracle.dsgrft_rows(sc.radar, s, sc.ds, cells, fine)
    assert np.array_equal(Ya, Y1) and np.array_equal(Ya, Yb)
