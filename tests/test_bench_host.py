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


def test_reference_arm_prints_the_contract_line(capsys):
    """bench.py --impl reference: one JSON line with the contract's keys, the oracle timed on
    the host (a tiny sample here)."""
    import argparse
    import json
    args = argparse.Namespace(gpus=1, steps=1, warmup=1, ref_step_s=0.2, ref_total_s=0.2)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]



def test_pd_trials_are_replayable_and_hit_rule():
    """Each Monte-Carlo trial is drawn from its own seed (replayable alone, distinct across
    trials and SNRs), its target lies off the grid's edges, and the hit rule accepts a
    detection within one cell of the truth on every axis and nothing farther."""
    R, ds, _, cf = synth.pd_setup()
    pg = ds.plain_equivalent()
    a = synth.pd_trial(R, pg, -10.0, 3)
    b = synth.pd_trial(R, pg, -10.0, 3)
    c = synth.pd_trial(R, pg, -10.0, 4)
    d = synth.pd_trial(R, pg, -12.0, 3)
    assert a[:3] == b[:3] and np.array_equal(a[3], b[3])
    assert not np.array_equal(a[3], c[3]) and not np.array_equal(a[3], d[3])
    j, k, n0, s = a
    assert 1 <= j < pg.v.count - 1 and 1 <= k < pg.a.count - 1 and 0 < n0 < R.N
    assert s.shape == (R.M, R.N) and s.dtype == np.complex64
    assert cf.mode == 1 and abs(cf.fixed_thresh + R.M * np.log(synth.PD_PFA)) < 1e-3
    assert bench.pd_hit([j + 1], [k - 1], [n0 + 1], j, k, n0)
    assert not bench.pd_hit([j + 2], [k], [n0], j, k, n0)
    assert not bench.pd_hit([], [], [], j, k, n0)
