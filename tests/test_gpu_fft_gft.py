"""GPU: the FFT form of the fine stage (Def. 1 / Alg. 2, dsgrft_fine_dfm_fft) on grids whose
fine velocity step is one Doppler bin of a 256- or 512-point transform, against the FP64
oracle's per-hypothesis DS-GRFT sums (every output of a small case with ragged tiles and a
cell sub-range; sampled rows at the M=512 x N=4096 shape) and against the dense
tensor-core contraction on the same hypotheses; grids it cannot serve are rejected."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.wrap import ds_rows_of_canonical
from synth import Axis, DSGrid, Radar, Target
from tests.helpers import TOL_FP32, TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu


def _fft_grid(R, L, Fv, vcount, ac, Fa, r0b, r0c):
    vstep_c = R.wavelength * R.prf_hz * Fv / (2 * L)     # Fv Doppler bins of an L-point transform
    return DSGrid(r0b, r0c, Axis(-(vcount // 2) * vstep_c, vstep_c, vcount), ac, Fv, Fa)


def test_fft_form_every_output_small(cuda_lib):
    g = cuda_lib
    R = Radar(M=200, N=600, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = _fft_grid(R, 256, 32, 4, Axis(-4.0, 4.0, 3), 4, 10, 500)
    s = synth.make_echo(R, [Target(300.0, 10.0, 2.0, complex(2.0, 1.0)),
                            Target(150.0, -20.0, -3.0, complex(0.5, -1.5))], 31)
    echo = torch.from_numpy(s).cuda()
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    Y = torch.zeros((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    P = torch.zeros((nv, na, ds.r0_count), device="cuda")
    g.dsgrft_fine_dfm_fft(R, echo, ds, 0, ds.n_cells, Y, P)
    assert g.grft_sync_status() == 0
    Yo = oracle.dsgrft_full(R, s, ds)
    Yg = Y.cpu().numpy()
    assert rel_peak_err(Yg, Yo) <= TOL_FP32
    np.testing.assert_allclose(P.cpu().numpy(), np.abs(Yg) ** 2, rtol=1e-5, atol=1e-6 * np.abs(Yg).max() ** 2)
    # a cell sub-range lands in its own v-slab; cells outside the range are untouched
    ac = ds.ac.count
    Ys = torch.full((ds.Fv, na, ds.r0_count), 7.0 + 0j, dtype=torch.complex64, device="cuda")
    g.dsgrft_fine_dfm_fft(R, echo, ds, ac + 1, ac - 1, Ys, None)
    ys = Ys.cpu().numpy()
    assert np.all(ys[:, :ds.Fa] == 7.0)
    assert rel_peak_err(ys[:, ds.Fa:], Yo[ds.Fv:2 * ds.Fv, ds.Fa:]) <= TOL_FP32


def test_fft_form_matches_oracle_and_dense_at_m512(cuda_lib):
    """M=512 x N=4096 radar, fine grid 96 x 16 (velocity step = one bin of a 512-point
    transform), every range bin of two coarse v rows: sampled rows against the oracle, the
    whole slab against the dense split-BF16 contraction."""
    g = cuda_lib
    sc = synth.ds_m512()
    R = sc.radar
    base = sc.ds
    ds = _fft_grid(R, 512, 96, base.vc.count, base.ac, base.Fa, 0, R.N)
    assert abs(ds.vc.step - base.vc.step) < 1e-12                 # the same coarse cells
    s = synth.make_echo(R, sc.targets, sc.seed)
    echo = torch.from_numpy(s).cuda()
    t = max(sc.targets, key=lambda t: abs(t.amp))
    i_row = min(max(int((t.v - (ds.vc.start - ds.vc.step / 2)) // ds.vc.step), 0), ds.vc.count - 2)
    cb, cc = i_row * ds.ac.count, 2 * ds.ac.count
    nv, na = 2 * ds.Fv, ds.ac.count * ds.Fa
    Yf = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    Yd = torch.empty_like(Yf)
    g.dsgrft_fine_dfm_fft(R, echo, ds, cb, cc, Yf, None)
    g.dsgrft_fine_dfm(R, None, echo, ds, cb, cc, "bf16x3", Yd, None)
    assert g.grft_sync_status() == 0
    yf, yd = Yf.cpu().numpy(), Yd.cpu().numpy()
    assert rel_peak_err(yf, yd) <= TOL_SPLIT
    rng = np.random.default_rng(2)
    vloc, af = rng.integers(0, nv, 8), rng.integers(0, na, 8)
    cell, fine = ds_rows_of_canonical(ds, vloc + i_row * ds.Fv, af)
    Yo = oracle.dsgrft_rows(R, s, ds, cell, fine)
    assert rel_peak_err(yf[vloc, af], Yo) <= TOL_FP32


def test_fft_form_rejects_grids_it_cannot_serve(cuda_lib):
    g = cuda_lib
    sc = synth.ds_m512()
    R, ds = sc.radar, sc.ds                       # fine step 18.75/64: not a bin of 256 or 512
    echo = torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda")
    P = torch.empty((ds.Fv, ds.ac.count * ds.Fa, ds.r0_count), device="cuda")
    with pytest.raises(g.GrftError):
        g.dsgrft_fine_dfm_fft(R, echo, ds, 0, ds.ac.count, None, P)
    odd = _fft_grid(R, 512, 96, 4, ds.ac, ds.Fa, 0, 64)
    odd = dataclasses.replace(odd, Fv=95)          # odd Fv
    with pytest.raises(g.GrftError):
        g.dsgrft_fine_dfm_fft(R, echo, odd, 0, 1, None, P)
    big_m = dataclasses.replace(R, M=600)          # more pulses than the transform
    with pytest.raises(g.GrftError):
        g.dsgrft_fine_dfm_fft(big_m, torch.zeros((600, R.N), dtype=torch.complex64, device="cuda"),
                              _fft_grid(big_m, 512, 96, 4, ds.ac, ds.Fa, 0, 64), 0, 1, None, P)
    assert g.grft_sync_status() == 0
