"""GPU parity: trajectory tables (bit-exact bins) and plain GRFT vs the FP64 oracle,
through the C ABI."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Axis, PlainGrid, Radar, Target
from tests.helpers import TOL_FP32, rel_peak_err

pytestmark = pytest.mark.gpu


def test_bins_bit_exact_and_phases(cuda_lib):
    g = cuda_lib
    R = Radar(M=512, N=4096, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    rng = np.random.default_rng(0)
    v = rng.uniform(-400, 400, 3000)
    a = rng.uniform(-30, 30, 3000)
    # exact half-bin ties (dyadic PRF) appended on a second radar below
    rho_o, w_o = oracle.bins_phases(R, v, a)
    vt, at = torch.tensor(v, device="cuda"), torch.tensor(a, device="cuda")
    rho = torch.empty((v.size, R.M), dtype=torch.int32, device="cuda")
    w = torch.empty((v.size, R.M), dtype=torch.complex64, device="cuda")
    g.grft_bins_phases(R, vt, at, rho, w)
    assert np.array_equal(rho.cpu().numpy(), rho_o)
    assert np.abs(w.cpu().numpy() - w_o).max() < 2e-6
    # ties: v = +-7680 m/s at PRF 1024 Hz put d exactly on half bins
    R2 = Radar(M=8, N=64, fc_hz=1.0e9, prf_hz=1024.0, dr_m=15.0)
    vt = torch.tensor([7680.0, -7680.0, 3840.0], dtype=torch.float64, device="cuda")
    at = torch.zeros(3, dtype=torch.float64, device="cuda")
    rho = torch.empty((3, 8), dtype=torch.int32, device="cuda")
    w = torch.empty((3, 8), dtype=torch.complex64, device="cuda")
    g.grft_bins_phases(R2, vt, at, rho, w)
    ro, _ = oracle.bins_phases(R2, vt.cpu().numpy(), at.cpu().numpy())
    assert np.array_equal(rho.cpu().numpy(), ro)
    assert ro[0].tolist() == [0, 1, 1, 2, 2, 3, 3, 4]


def _plain_case(R, grid, s):
    g = pytest.importorskip("paper_2403_06788_gb300")
    es = torch.from_numpy(s).cuda()
    P, Y = g.grft(R, es, grid, want_Y=True)
    Yo = oracle.grft_plain_full(R, s, grid)
    return P.cpu().numpy(), Y.cpu().numpy(), Yo


def test_plain_m64_full_grid(cuda_lib):
    """plain_m64: M=64, N=256, one target, 256 x 64 x 16 hypotheses, every output compared."""
    sc = synth.plain_m64()
    s = synth.make_echo(sc.radar, sc.targets, sc.seed)
    P, Y, Yo = _plain_case(sc.radar, sc.plain, s)
    assert rel_peak_err(Y, Yo) <= TOL_FP32
    assert rel_peak_err(P, np.abs(Yo) ** 2) <= 2 * TOL_FP32
    # the peak is at the target's grid cell
    vi, ai, n0 = np.unravel_index(P.argmax(), P.shape)
    assert (vi, ai) == (32, 8) and abs(n0 - 100) <= 1


@pytest.mark.parametrize("M,N,r0b,r0c,nv,na", [
    (37, 700, 5, 1500 - 803, 11, 3),     # ragged M, r0 sub-range, tail tile, partial hyp group
    (1, 64, 0, 64, 3, 2),                # single pulse
    (200, 300, 250, 50, 9, 9),           # r0 window near the top edge (bins leave [0, N))
])
def test_plain_ragged_and_edges(cuda_lib, M, N, r0b, r0c, nv, na):
    R = Radar(M=M, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    r0c = min(r0c, N - r0b)
    grid = PlainGrid(r0b, r0c, Axis(-280.0, 61.3, nv), Axis(-18.0, 4.4, na))
    s = synth.make_echo(R, [Target(N / 2, 50.0, 3.0, complex(2.0, 1.0))], 7 + M)
    P, Y, Yo = _plain_case(R, grid, s)
    assert rel_peak_err(Y, Yo) <= TOL_FP32


def test_plain_rejects_bad_arguments(cuda_lib):
    g = cuda_lib
    sc = synth.plain_m64()
    es = torch.zeros((sc.radar.M, sc.radar.N), dtype=torch.complex64, device="cuda")
    P = torch.empty(10, device="cuda")
    bad = dataclasses.replace(sc.plain, r0_begin=200, r0_count=100)    # beyond N
    with pytest.raises(g.GrftError) as ei:
        g.grft_plain(sc.radar, es, bad, None, P)
    assert ei.value.code == -1
    with pytest.raises(g.GrftError):
        g.grft_plain(sc.radar, es, sc.plain, None, None)               # no output
