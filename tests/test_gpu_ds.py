"""GPU parity of the DS-GRFT path (coarse RM gather, fine DFM contraction in FP32 SIMT and
on the tensor cores in split BF16/FP16, two-product split FP16 and single-product FP16)
against the FP64 oracle, through the C ABI."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Axis, DSGrid, Radar, Target
from tests.helpers import TOL_FP32, TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu

TOL = {"fp32": TOL_FP32, "bf16x3": TOL_SPLIT, "fp16x3": TOL_SPLIT, "fp16x2": TOL_SPLIT, "fp16x1": TOL_SPLIT}


def _small_case(M=100, N=700, r0b=17, r0c=300, Fv=16, Fa=16, nvc=3, nac=2, seed=3):
    """Spans several tiles and ragged tails on every axis: 3 bin tiles (last partial),
    2 fine-hypothesis tiles, 4 pulse stages (last partial), 6 coarse cells."""
    R = Radar(M=M, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(r0b, r0c, Axis(-40.0, 18.75, nvc), Axis(-2.5, 5.0, nac), Fv, Fa)
    tg = [Target(r0b + 120.0, -21.0, 1.2, complex(3.0, -1.0)), Target(r0b + 251.3, 3.0, -2.0, complex(1.0, 2.0))]
    s = synth.make_echo(R, tg, seed)
    return R, ds, s


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16x3", "fp16x2", "fp16x1"])
def test_ds_fused_small_every_output(cuda_lib, precision):
    g = cuda_lib
    R, ds, s = _small_case()
    es = torch.from_numpy(s).cuda()
    P, Y = g.dsgrft(R, es, ds, precision=precision, want_Y=True)
    assert g.grft_sync_status() == 0
    Yo = oracle.dsgrft_full(R, s, ds)
    err = rel_peak_err(Y.cpu().numpy(), Yo)
    assert err <= TOL[precision], err
    assert rel_peak_err(P.cpu().numpy(), np.abs(Yo) ** 2) <= 2 * TOL[precision]
    if precision in ("bf16x3", "fp16x3"):
        # the split path is far better than its 2e-3 bound; guard against silent regressions
        assert err <= 1e-4, err
    if precision in ("fp16x2", "fp16x1"):
        # one FP16 rounding of the dechirp (and, for fp16x1, of the echo operand): about
        # 2^-12 per term, well inside the 2e-3 bound
        assert err <= 5e-4, err


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ds_with_materialised_Z_matches_fused(cuda_lib, precision):
    g = cuda_lib
    R, ds, s = _small_case(seed=4)
    es = torch.from_numpy(s).cuda()
    Yf = g.dsgrft(R, es, ds, precision=precision, want_Y=True, want_P=False)
    Yz = g.dsgrft(R, es, ds, precision=precision, want_Y=True, want_P=False, fused=False)
    assert rel_peak_err(Yz.cpu().numpy(), Yf.cpu().numpy()) <= 1e-6


def test_coarse_rm_matches_oracle(cuda_lib):
    g = cuda_lib
    for N in (700, 701):            # even N takes the TMA path, odd N the plain-load path
        R, ds, s = _small_case(N=N)
        es = torch.from_numpy(s).cuda()
        ncell = ds.n_cells
        Z = torch.empty((ncell, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
        g.dsgrft_coarse_rm(R, es, ds, 0, ncell, Z)
        Zo = oracle.coarse_rm(R, s, ds, 0, ncell)
        assert rel_peak_err(Z.cpu().numpy(), Zo) <= 1e-6
        # bins are exact: the zero pattern (samples gathered from outside [0, N)) matches
        assert np.array_equal(Z.cpu().numpy() == 0, Zo == 0)


def test_coarse_rm_cell_subrange_and_edges(cuda_lib):
    g = cuda_lib
    R = Radar(M=50, N=256, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    # fast coarse velocities push the gathered bins off both ends of the echo
    ds = DSGrid(0, 256, Axis(-300.0, 150.0, 5), Axis(-20.0, 40.0, 2), 4, 2)
    s = synth.make_noise((R.M, R.N), 9)
    es = torch.from_numpy(s).cuda()
    Z = torch.empty((3, R.M, 256), dtype=torch.complex64, device="cuda")
    g.dsgrft_coarse_rm(R, es, ds, 4, 3, Z)
    Zo = oracle.coarse_rm(R, s, ds, 4, 3)
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= 1e-6


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ds_cell_slab_output_layout(cuda_lib, precision):
    """A call over cells [cell_begin, +count) writes the v-slab of the canonical layout and
    leaves other cells untouched."""
    g = cuda_lib
    R, ds, s = _small_case(nvc=4, nac=3)
    es = torch.from_numpy(s).cuda()
    nac, Fv, Fa = ds.ac.count, ds.Fv, ds.Fa
    cb, cc = 4, 5                     # cells 4..8 -> coarse v rows 1..2
    i0, i1 = cb // nac, (cb + cc - 1) // nac
    P = torch.full(((i1 - i0 + 1) * Fv, nac * Fa, ds.r0_count), -1.0, device="cuda")
    g.dsgrft_fine_dfm(R, None, es, ds, cb, cc, precision, None, P)
    Pn = P.cpu().numpy()
    Pfull = np.abs(oracle.dsgrft_full(R, s, ds)) ** 2
    for c in range(cb, cb + cc):
        i, l = divmod(c, nac)
        blk = Pn[(i - i0) * Fv:(i - i0 + 1) * Fv, l * Fa:(l + 1) * Fa]
        ref = Pfull[i * Fv:(i + 1) * Fv, l * Fa:(l + 1) * Fa]
        assert rel_peak_err(blk, ref) <= 2 * TOL[precision]
    # cell 3 = (1, 0) precedes the range and stays untouched
    assert np.all(Pn[0:Fv, 0:Fa] == -1.0)


def test_ds_fine_grid_padding_and_single_cell(cuda_lib):
    """F = 5 x 3 = 15 fine hypotheses (padded to a 128-wide tile), one cell, M = 33."""
    g = cuda_lib
    R, ds, s = _small_case(M=33, Fv=5, Fa=3, nvc=1, nac=1, r0c=129)
    es = torch.from_numpy(s).cuda()
    for prec in ("fp32", "bf16x3", "fp16x3", "fp16x2", "fp16x1"):
        Y = g.dsgrft(R, es, ds, precision=prec, want_Y=True, want_P=False)
        assert rel_peak_err(Y.cpu().numpy(), oracle.dsgrft_full(R, s, ds)) <= TOL[prec]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x2", "fp16x1"])
def test_ds_long_cpi_tables_from_global_memory(cuda_lib, precision):
    """M = 2100 pulses: more than the operand-split kernel stages in shared memory (2048), so it
    reads the cell's bins and phases from global memory; 66 pulse stages, the last partial."""
    g = cuda_lib
    R, ds, s = _small_case(M=2100, N=400, r0b=5, r0c=260, Fv=4, Fa=2, nvc=2, nac=1, seed=6)
    es = torch.from_numpy(s).cuda()
    Y = g.dsgrft(R, es, ds, precision=precision, want_Y=True, want_P=False)
    assert g.grft_sync_status() == 0
    err = rel_peak_err(Y.cpu().numpy(), oracle.dsgrft_full(R, s, ds))
    assert err <= TOL[precision] and err <= (1e-4 if precision == "bf16x3" else 5e-4), err


def test_ds_full_ds_m512_sampled(cuda_lib):
    """ds_m512 at full size (2^30 hypotheses) in the launch configuration the benchmark times,
    compared with the oracle on sampled rows (every r0 of 24 (v, a) rows, incl. targets)."""
    g = cuda_lib
    sc = synth.ds_m512()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets, sc.seed)
    es = torch.from_numpy(s).cuda()
    pg = ds.plain_equivalent()
    rng = np.random.default_rng(11)
    vf = list(rng.integers(0, pg.v.count, 16))
    af = list(rng.integers(0, pg.a.count, 16))
    for t in sc.targets:
        vf.append(int(round((t.v - pg.v.start) / pg.v.step)))
        af.append(int(round((t.a - pg.a.start) / pg.a.step)))
    vf, af = np.clip(vf, 0, pg.v.count - 1), np.clip(af, 0, pg.a.count - 1)
    from oracle.wrap import ds_rows_of_canonical
    cell, fine = ds_rows_of_canonical(ds, vf, af)
    Yo = oracle.dsgrft_rows(R, s, ds, cell, fine)
    for prec in ("bf16x3", "fp16x2", "fp32", "fp16x1"):
        Y = g.dsgrft(R, es, ds, precision=prec, want_Y=True, want_P=False)
        assert g.grft_sync_status() == 0
        Yg = Y[torch.as_tensor(vf, device="cuda"), torch.as_tensor(af, device="cuda")].cpu().numpy()
        err = rel_peak_err(Yg, Yo)
        print(prec, "max rel peak error on sampled rows:", err)
        assert err <= TOL[prec]
        del Y
        torch.cuda.empty_cache()
