"""GPU: the frequency-domain coarse stage (mGIFT with H_RM as a range-spectrum ramp, Alg. 1,
dsgrft_coarse_rm_fd) against the FP64 numpy oracle (every output of a small case with a
ragged range window; sampled pulses at M=512 x N=4096), the fine stage run on its output
(dsgrft_fine_dfm with Z given) against the oracle's DS-GRFT rows of the same form, the
paper's positive band (asinc echo, k = 0..N-1) with the fine-offset scale of Prop. 1, and
the rejection of range lengths that are not a power of two."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Axis, DSGrid, Radar, Target
from tests.helpers import TOL_FP32, TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu


def _small():
    R = Radar(M=64, N=256, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(5, 200, Axis(-120.0, 60.0, 3), Axis(-10.0, 20.0, 2), 4, 2)
    s = synth.make_echo(R, [Target(90.3, -70.0, 6.0, complex(3.0, -1.0)),
                            Target(170.6, 40.0, -4.0, complex(-1.0, 2.0))], 17)
    return R, ds, s


def test_fd_coarse_stage_every_output_small(cuda_lib):
    g = cuda_lib
    R, ds, s = _small()
    Z = torch.zeros((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd(R, torch.from_numpy(s).cuda(), ds, 0, ds.n_cells, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.coarse_rm_fd(R, s, ds, 0, ds.n_cells)
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32
    # a cell sub-range: the same values for those cells
    Zs = torch.zeros((2, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd(R, torch.from_numpy(s).cuda(), ds, 3, 2, Zs)
    assert rel_peak_err(Zs.cpu().numpy(), Zo[3:5]) <= TOL_FP32


@pytest.mark.parametrize("N", [128, 512, 1024, 2048])
def test_fd_coarse_stage_every_output_all_pass_shapes(cuda_lib, N):
    """Range lengths whose log2 leaves 3, 1, 2 and 3 stages for the last pass of the
    shared-memory transforms (passes of up to four radix-2 stages), both bands."""
    g = cuda_lib
    R = Radar(M=24, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(3, N - 9, Axis(-150.0, 100.0, 3), Axis(-10.0, 20.0, 1), 2, 1)
    s = synth.make_echo(R, [Target(0.45 * N, -60.0, 4.0, complex(2.0, -1.0))], 40 + N % 97)
    for band in ("baseband", "positive"):
        Z = torch.zeros((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
        g.dsgrft_coarse_rm_fd_ex(R, torch.from_numpy(s).cuda(), ds, 0, ds.n_cells, band, Z)
        assert g.grft_sync_status() == 0
        Zo = oracle.coarse_rm_fd(R, s, ds, 0, ds.n_cells, band=band)
        assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32, band


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("bf16x3", TOL_SPLIT)])
def test_fd_then_fine_stage_matches_oracle_rows(cuda_lib, precision, tol):
    g = cuda_lib
    R, ds, s = _small()
    echo = torch.from_numpy(s).cuda()
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd(R, echo, ds, 0, ds.n_cells, Z)
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_fine_dfm(R, Z, echo, ds, 0, ds.n_cells, precision, Y, None)
    assert g.grft_sync_status() == 0
    vf, af = np.meshgrid(np.arange(nv), np.arange(na), indexing="ij")
    from oracle.wrap import ds_rows_of_canonical
    cell, fine = ds_rows_of_canonical(ds, vf.ravel(), af.ravel())
    Yo = oracle.dsgrft_rows_fd(R, s, ds, cell, fine).reshape(nv, na, ds.r0_count)
    assert rel_peak_err(Y.cpu().numpy(), Yo) <= tol


def test_fd_coarse_stage_m512_sampled(cuda_lib):
    g = cuda_lib
    sc = synth.ds_m512()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets, sc.seed)
    cb, cc = 100, 4
    Z = torch.empty((cc, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd(R, torch.from_numpy(s).cuda(), ds, cb, cc, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.coarse_rm_fd(R, s, ds, cb, cc)
    ms = np.random.default_rng(5).integers(0, R.M, 24)
    assert rel_peak_err(Z.cpu().numpy()[:, ms], Zo[:, ms]) <= TOL_FP32


def test_fd_coarse_stage_rejects_non_power_of_two(cuda_lib):
    g = cuda_lib
    R = Radar(M=16, N=300, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(0, 100, Axis(0.0, 10.0, 1), Axis(0.0, 1.0, 1), 2, 2)
    Z = torch.empty((1, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    with pytest.raises(g.GrftError):
        g.dsgrft_coarse_rm_fd(R, torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda"), ds, 0, 1, Z)
    assert g.grft_sync_status() == 0


def _small_asinc():
    R = Radar(M=64, N=256, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(5, 200, Axis(-120.0, 60.0, 3), Axis(-10.0, 20.0, 2), 4, 2)
    s = synth.make_echo(R, [Target(90.3, -70.0, 6.0, complex(3.0, -1.0)),
                            Target(170.6, 40.0, -4.0, complex(-1.0, 2.0))], 18, envelope="asinc")
    return R, ds, s


def test_fd_coarse_stage_positive_band_every_output(cuda_lib):
    """The paper's band (k = 0..N-1, eq. Rx-OFDM-Fre1) on an asinc echo, every output."""
    g = cuda_lib
    R, ds, s = _small_asinc()
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd_ex(R, torch.from_numpy(s).cuda(), ds, 0, ds.n_cells, "positive", Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.coarse_rm_fd(R, s, ds, 0, ds.n_cells, band="positive")
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32
    Zb = oracle.coarse_rm_fd(R, s, ds, 0, ds.n_cells)                 # the other reading differs
    assert rel_peak_err(Zb, Zo) > 1e-3


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("bf16x3", TOL_SPLIT)])
def test_fd_positive_band_fine_stage_with_fine_scale(cuda_lib, precision, tol):
    """Positive-band coarse stage, then the fine stage with the fine offsets scaled by
    1 + B_r / (2 f_c) (dsgrft_fine_dfm_fd), against the oracle's rows, every output."""
    g = cuda_lib
    R, ds, s = _small_asinc()
    P, Y = g.dsgrft_fd(R, torch.from_numpy(s).cuda(), ds, band="positive", precision=precision, want_Y=True)
    assert g.grft_sync_status() == 0
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    vf, af = np.meshgrid(np.arange(nv), np.arange(na), indexing="ij")
    from oracle.wrap import ds_rows_of_canonical
    cell, fine = ds_rows_of_canonical(ds, vf.ravel(), af.ravel())
    Yo = oracle.dsgrft_rows_fd(R, s, ds, cell, fine, band="positive",
                               kap=oracle.fine_scale(R, "positive")).reshape(nv, na, ds.r0_count)
    assert rel_peak_err(Y.cpu().numpy(), Yo) <= tol
    # baseband: the same entry points give the unscaled form
    Pb, Yb = g.dsgrft_fd(R, torch.from_numpy(s).cuda(), ds, band="baseband", precision=precision, want_Y=True)
    Yob = oracle.dsgrft_rows_fd(R, s, ds, cell, fine).reshape(nv, na, ds.r0_count)
    assert rel_peak_err(Yb.cpu().numpy(), Yob) <= tol


def test_fd_positive_band_m512_sampled(cuda_lib):
    g = cuda_lib
    sc = synth.ds_m512()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets[:3], sc.seed, envelope="asinc")
    cb, cc = 77, 3
    Z = torch.empty((cc, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm_fd_ex(R, torch.from_numpy(s).cuda(), ds, cb, cc, "positive", Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.coarse_rm_fd(R, s, ds, cb, cc, band="positive")
    ms = np.random.default_rng(9).integers(0, R.M, 24)
    assert rel_peak_err(Z.cpu().numpy()[:, ms], Zo[:, ms]) <= TOL_FP32
