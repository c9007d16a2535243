"""GPU: per-kernel CUDA-event timing through the C ABI (grft_timing / grft_timing_get).
Counts must equal the launches each call makes, times must be positive and bounded by the
host wall clock, and a call inside stream capture records nothing."""
import time

import pytest
import torch

import synth
from synth import Axis, DSGrid, Radar, Target

pytestmark = pytest.mark.gpu


def _case():
    R = Radar(M=128, N=1024, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(0, 1024, Axis(-40.0, 18.75, 2), Axis(-2.5, 5.0, 2), 16, 8)
    s = synth.make_echo(R, [Target(4000.0, -20.0, 1.0, complex(3.0, 0.0))], 3)
    return R, ds, torch.from_numpy(s).cuda()


def test_timing_counts_and_totals(cuda_lib):
    g = cuda_lib
    R, ds, echo = _case()
    g.dsgrft(R, echo, ds, precision="bf16x3")          # warm-up: workspace, autotune
    torch.cuda.synchronize()
    g.grft_timing(True)
    t0 = time.perf_counter()
    n_calls = 3
    for _ in range(n_calls):
        g.dsgrft(R, echo, ds, precision="bf16x3")
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    n_split, ms_split = g.grft_timing_get("split")
    n_ctr, ms_ctr = g.grft_timing_get("contract")
    n_plain, ms_plain = g.grft_timing_get("plain")
    assert n_split >= n_calls and n_ctr == n_split           # one contraction per split round
    assert 0.0 < ms_split < wall_ms and 0.0 < ms_ctr < wall_ms
    assert n_plain == 0 and ms_plain == 0.0
    # disabling clears and stops recording
    g.grft_timing(False)
    g.dsgrft(R, echo, ds, precision="bf16x3")
    assert g.grft_timing_get("contract") == (0, 0.0)
    assert g.grft_sync_status() == 0


def test_timing_skips_captured_launches(cuda_lib):
    g = cuda_lib
    R, ds, echo = _case()
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    P = torch.empty((nv, na, ds.r0_count), device="cuda")
    g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.vc.count * ds.ac.count, "bf16x3", None, P)
    torch.cuda.synchronize()
    g.grft_timing(True)
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.vc.count * ds.ac.count, "bf16x3", None, P)
    graph.replay()
    torch.cuda.synchronize()
    assert g.grft_timing_get("contract") == (0, 0.0)
    g.grft_timing(False)
    assert g.grft_sync_status() == 0


def test_shutdown_releases_and_the_next_call_sets_up_again(cuda_lib):
    g = cuda_lib
    R, ds, echo = _case()
    ref = g.dsgrft(R, echo, ds, precision="bf16x3")
    g.grft_timing(True)
    g.dsgrft(R, echo, ds, precision="bf16x3")
    g.grft_shutdown()                                  # also drops pending timing events
    again = g.dsgrft(R, echo, ds, precision="bf16x3")
    assert torch.equal(ref, again)
    assert g.grft_timing_get("contract") == (0, 0.0)    # timing is off after shutdown
    assert g.grft_sync_status() == 0
