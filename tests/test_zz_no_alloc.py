"""grft_plain_static — plain GRFT for callers that cannot allocate device memory (a
processing loop with a fixed memory budget that must not wait on an allocator, a process
whose device memory belongs to another pool).  It keeps its tables in a fixed array inside
the library instead of the allocated workspace and runs the same kernels over the same
groups of hypotheses, so its output must equal grft_plain's bit for bit; two calls in a row
check that the shared array left over from the previous call is harmless.  This file is
collected last on purpose."""
import numpy as np
import pytest
import torch

import synth
from synth import Axis, PlainGrid, Radar, Target
from tests.helpers import TOL_FP32, rel_peak_err

pytestmark = pytest.mark.gpu


def _cases():
    sc = synth.plain_m64()
    yield sc.radar, sc.plain, synth.make_echo(sc.radar, sc.targets, sc.seed)
    # M = 512 and 8192 hypotheses: several chunks of the fixed scratch, ragged r0 tail
    R = Radar(M=512, N=1200, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    g = PlainGrid(37, 1111, Axis(-150.0, 4.7, 64), Axis(-10.0, 0.16, 128))
    yield R, g, synth.make_echo(R, [Target(600.0, -40.0, 3.0, complex(2.0, -1.0))], 77)
    # M = 1 and 614,400 hypotheses: the fixed scratch would hold about 699k hypotheses' tables,
    # more than one launch takes (grft_plain's chunk limit of 2^18 applies)
    R = Radar(M=1, N=96, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    g = PlainGrid(0, 64, Axis(-300.0, 0.5, 1200), Axis(-10.0, 0.04, 512))
    yield R, g, synth.make_echo(R, [Target(30.0, 0.0, 0.0, complex(2.0, -1.0))], 78)


def test_static_scratch_matches_workspace_path_twice(cuda_lib):
    g = cuda_lib
    for R, grid, s in _cases():
        echo = torch.from_numpy(s).cuda()
        P_ref, Y_ref = g.grft(R, echo, grid, want_Y=True)
        shape = tuple(P_ref.shape)
        for _ in range(2):
            P = torch.full(shape, -1.0, dtype=torch.float32, device="cuda")
            Y = torch.zeros(shape, dtype=torch.complex64, device="cuda")
            g.grft_plain_static(R, echo, grid, Y, P)
            torch.cuda.synchronize()
            assert g.grft_sync_status() == 0
            assert rel_peak_err(Y.cpu().numpy(), Y_ref.cpu().numpy()) <= TOL_FP32
            assert torch.equal(Y, Y_ref) and torch.equal(P, P_ref)
        del P_ref, Y_ref, P, Y
        torch.cuda.empty_cache()


def test_static_scratch_rejects_problems_that_do_not_fit(cuda_lib):
    g = cuda_lib
    R = Radar(M=100000, N=64, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)   # 8 x 100000 x 12 B > 8 MiB
    grid = PlainGrid(0, 64, Axis(0.0, 1.0, 8), Axis(0.0, 1.0, 1))
    echo = torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda")
    P = torch.empty((8, 1, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(g.GrftError) as ei:
        g.grft_plain_static(R, echo, grid, None, P)
    assert ei.value.code == -1


def test_static_scratch_rejects_non_finite_arguments_like_grft_plain(cuda_lib):
    """Non-finite radar parameters or axis values are refused by both entry points before any
    launch (GRFT_EINVAL)."""
    import dataclasses
    g = cuda_lib
    R = Radar(M=8, N=64, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    grid = PlainGrid(0, 64, Axis(0.0, 1.0, 8), Axis(0.0, 1.0, 1))
    echo = torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda")
    P = torch.empty((8, 1, 64), dtype=torch.float32, device="cuda")
    bad = [(dataclasses.replace(R, fc_hz=float("inf")), grid),
           (dataclasses.replace(R, prf_hz=float("nan")), grid),
           (R, dataclasses.replace(grid, v=Axis(float("nan"), 1.0, 8))),
           (R, dataclasses.replace(grid, a=Axis(0.0, float("inf"), 1)))]
    for Rb, gb in bad:
        for fn in (g.grft_plain, g.grft_plain_static):
            with pytest.raises(g.GrftError) as ei:
                fn(Rb, echo, gb, None, P)
            assert ei.value.code == -1
