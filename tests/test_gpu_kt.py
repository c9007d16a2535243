"""GPU: the keystone branch, DS-KT-MFP (eq. Echo-after-KT, Cor. 1, Prop. 3, Alg. 4), through
the C ABI against the FP64 numpy oracle: the keystone transform (every output of small
cases, sampled columns at M=512 x N=4096 and M=2048), the H_KT,RM coarse stage and the
FFT-form fine stage (every output of small cases with a ragged range window and a
zero-padded transform; sampled outputs at full size, from seeded synthetic inputs), the
whole map (every output of a small case), target focus on the 1.88e9-hypothesis grid, and
the rejection of unsupported sizes and grids."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Axis, DSGrid, Radar, Target
from tests.helpers import TOL_FP32, rel_peak_err

pytestmark = pytest.mark.gpu


def _slots(g, N):
    return np.asarray(g.spectral_slots(N))


def _keystone(g, R, s):
    Skt = torch.empty((R.M, R.N), dtype=torch.complex64, device="cuda")
    g.dskt_keystone(R, torch.from_numpy(s).cuda(), Skt)
    assert g.grft_sync_status() == 0
    return Skt.cpu().numpy()


@pytest.mark.parametrize("M,N", [(64, 256), (16, 4), (128, 64), (1024, 32)])
def test_keystone_every_output(cuda_lib, M, N):
    g = cuda_lib
    R = Radar(M=M, N=N, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    s = synth.make_echo(R, [Target(N * 0.4, 120.0, 5.0, complex(2.0, 1.0))], 31)
    got = _keystone(g, R, s)
    want = oracle.keystone(R, s)[:, _slots(g, N)]
    assert rel_peak_err(got, want) <= TOL_FP32


@pytest.mark.parametrize("M,N,ncol", [(512, 4096, 24), (2048, 64, 6)])
def test_keystone_sampled_columns(cuda_lib, M, N, ncol):
    g = cuda_lib
    R = Radar(M=M, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    s = synth.make_echo(R, [Target(N * 0.3, 250.0, -8.0, complex(1.0, -3.0))], 32)
    got = _keystone(g, R, s)
    slots = _slots(g, N)
    ps = np.concatenate([[0, 1, N - 1], np.random.default_rng(3).integers(0, N, ncol - 3)])
    want = oracle.keystone_columns(R, s, slots[ps])
    assert rel_peak_err(got[:, ps], want) <= TOL_FP32


def _small_kt():
    R = Radar(M=64, N=256, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    ds = synth.kt_grid(R, -2, 5, Axis(-15.0, 10.0, 4), 4, r0_begin=7, r0_count=201)
    return R, ds


def test_kt_coarse_stage_every_output(cuda_lib):
    g = cuda_lib
    R, ds = _small_kt()
    ykt = synth.make_noise((R.M, R.N), 41).astype(np.complex128)
    Skt = torch.from_numpy(np.ascontiguousarray(ykt[:, _slots(g, R.N)].astype(np.complex64))).cuda()
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, Skt, ds, 0, ds.n_cells, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.kt_coarse_rm(R, ykt.astype(np.complex64), ds, 0, ds.n_cells)
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32
    Zs = torch.empty((3, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, Skt, ds, 9, 3, Zs)
    assert rel_peak_err(Zs.cpu().numpy(), Zo[9:12]) <= TOL_FP32


@pytest.mark.parametrize("N", [128, 1024])
def test_kt_coarse_stage_every_output_all_pass_shapes(cuda_lib, N):
    """Range lengths whose log2 leaves 3 and 2 stages for the last pass of the inverse
    transform (passes of up to four radix-2 stages)."""
    g = cuda_lib
    R = Radar(M=32, N=N, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    ds = synth.kt_grid(R, -2, 3, Axis(-15.0, 10.0, 2), 2, r0_begin=5, r0_count=N - 11)
    ykt = synth.make_noise((R.M, R.N), 43 + N % 89).astype(np.complex128)
    Skt = torch.from_numpy(np.ascontiguousarray(ykt[:, _slots(g, R.N)].astype(np.complex64))).cuda()
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, Skt, ds, 0, ds.n_cells, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.kt_coarse_rm(R, ykt.astype(np.complex64), ds, 0, ds.n_cells)
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32


@pytest.mark.parametrize("L", [64, 128])
def test_kt_fine_stage_every_output(cuda_lib, L):
    g = cuda_lib
    R, ds = _small_kt()
    ds = dataclasses.replace(ds, Fv=L)
    Zn = synth.make_noise((ds.n_cells, R.M, ds.r0_count), 42)
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    P = torch.empty((nv, na, ds.r0_count), dtype=torch.float32, device="cuda")
    g.dskt_fine_dfm_fft(R, torch.from_numpy(Zn).cuda(), ds, 0, ds.n_cells, Y, P)
    assert g.grft_sync_status() == 0
    Yg = Y.cpu().numpy()
    fine = np.arange(ds.Fv * ds.Fa)
    for c in range(ds.n_cells):
        i, l = divmod(c, ds.ac.count)
        Yo = oracle.kt_fine_rows(R, Zn[c].astype(np.complex128), ds, fine).reshape(ds.Fv, ds.Fa, ds.r0_count)
        got = Yg[i * ds.Fv:(i + 1) * ds.Fv, l * ds.Fa:(l + 1) * ds.Fa]
        assert rel_peak_err(got, Yo) <= TOL_FP32, c
    assert np.allclose(P.cpu().numpy(), np.abs(Yg) ** 2, rtol=1e-5, atol=1e-6 * float(P.max()))


def test_dskt_map_every_output_small(cuda_lib):
    g = cuda_lib
    sc = synth.dskt_m64()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets, sc.seed)
    P, Y = g.dsktmfp(R, torch.from_numpy(s).cuda(), ds, want_Y=True)
    assert g.grft_sync_status() == 0
    Yo = oracle.dskt_map(R, s, ds)
    assert rel_peak_err(Y.cpu().numpy(), Yo) <= TOL_FP32
    # the three entry points in sequence give the same map
    Skt = torch.empty((R.M, R.N), dtype=torch.complex64, device="cuda")
    g.dskt_keystone(R, torch.from_numpy(s).cuda(), Skt)
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, Skt, ds, 0, ds.n_cells, Z)
    Y2 = torch.empty_like(Y)
    g.dskt_fine_dfm_fft(R, Z, ds, 0, ds.n_cells, Y2, None)
    assert torch.equal(Y2, Y)
    # each target peaks within one bin of its (r0, v, a)
    pg = ds.plain_equivalent()
    Pn = P.cpu().numpy()
    for t in sc.targets:
        iv = int(round((t.v - pg.v.start) / pg.v.step))
        ia = int(round((t.a - pg.a.start) / pg.a.step))
        ir = int(round(t.r0_bins)) - ds.r0_begin
        box = Pn[max(iv - 1, 0):iv + 2, max(ia - 1, 0):ia + 2, max(ir - 1, 0):ir + 2]
        assert box.max() >= 0.2 * (abs(t.amp) * R.M) ** 2, t


def test_kt_stages_full_size_sampled(cuda_lib):
    """M=512, N=4096 (the dskt_m512 radar): the coarse stage from a seeded synthetic post-KT
    spectrum and the fine stage from a seeded synthetic coarse output, sampled outputs."""
    g = cuda_lib
    sc = synth.dskt_m512()
    R, ds = sc.radar, sc.ds
    ykt = synth.make_noise((R.M, R.N), 43)
    Skt = torch.from_numpy(ykt[:, _slots(g, R.N)].copy()).cuda()
    cb, cc = 2 * ds.ac.count + 5, 3                      # q = -1, three a cells
    Z = torch.empty((cc, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, Skt, ds, cb, cc, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.kt_coarse_rm(R, ykt, ds, cb, cc)
    ms = np.random.default_rng(6).integers(0, R.M, 24)
    assert rel_peak_err(Z.cpu().numpy()[:, ms], Zo[:, ms]) <= TOL_FP32
    del Skt, Z
    # fine stage on one coarse row (all a cells of q = 1)
    i_row = 4
    Zn = synth.make_noise((ds.ac.count, R.M, ds.r0_count), 44)
    nv, na = ds.Fv, ds.ac.count * ds.Fa
    Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_fine_dfm_fft(R, torch.from_numpy(Zn).cuda(), ds, i_row * ds.ac.count, ds.ac.count, Y, None)
    assert g.grft_sync_status() == 0
    rng = np.random.default_rng(7)
    for l in (0, 5):
        fine = np.concatenate([[0, ds.Fv * ds.Fa - 1], rng.integers(0, ds.Fv * ds.Fa, 30)])
        Yo = oracle.kt_fine_rows(R, Zn[l].astype(np.complex128), ds, fine)
        k, q = np.divmod(fine, ds.Fa)
        got = Y[torch.as_tensor(k, device="cuda"), torch.as_tensor(l * ds.Fa + q, device="cuda")].cpu().numpy()
        assert rel_peak_err(got, Yo) <= TOL_FP32


def test_dskt_m512_focuses_every_target(cuda_lib):
    """The whole DS-KT-MFP map on the 8-target M=512 echo (SNR -13 to -3 dB per sample):
    every target's power is focused within one range bin and two fine velocity and
    acceleration bins of its motion (at least 0.2 (|A| M)^2: the straddle losses of an
    off-grid target stay above that, a walk over the folding factor's blind speed does
    not), and the three strongest targets are among the CFAR detections (CA-CFAR + local
    maximum) at those cells."""
    g = cuda_lib
    sc = synth.dskt_m512()
    R, ds = sc.radar, sc.ds
    pg = ds.plain_equivalent()
    s = synth.make_echo(R, sc.targets, sc.seed)
    P = g.dsktmfp(R, torch.from_numpy(s).cuda(), ds)
    assert g.grft_sync_status() == 0
    assert P.shape == (7 * 512, 128, 4096)
    for t in sc.targets:
        iv = int(round((t.v - pg.v.start) / pg.v.step))
        ia = int(round((t.a - pg.a.start) / pg.a.step))
        ir = int(round(t.r0_bins))
        box = P[max(iv - 2, 0):iv + 3, max(ia - 2, 0):ia + 3, max(ir - 1, 0):ir + 2]
        assert float(box.max()) >= 0.2 * (abs(t.amp) * R.M) ** 2, t
    out, n_out = g.detect_peaks(P, synth.CFAR(2, 16, 1e-6), 1000, axes=pg, dr_m=R.dr_m)
    dets, total = g.decode_detections(out, n_out, 1000)
    del P
    torch.cuda.empty_cache()
    for t in sorted(sc.targets, key=lambda t: -abs(t.amp))[:3]:
        ok = ((np.abs(dets["r0_m"] / R.dr_m - t.r0_bins) <= 1.0) & (np.abs(dets["v"] - t.v) <= 2 * pg.v.step)
              & (np.abs(dets["a"] - t.a) <= 2 * pg.a.step))
        assert ok.any(), (t, total)


def test_kt_rejects_unsupported(cuda_lib):
    g = cuda_lib
    R = Radar(M=100, N=256, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    echo = torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(g.GrftError):
        g.dskt_keystone(R, echo, torch.empty_like(echo))
    R = Radar(M=64, N=256, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    ok = synth.kt_grid(R, -1, 3, Axis(0.0, 10.0, 1), 2)
    Z = torch.zeros((3, R.M, R.N), dtype=torch.complex64, device="cuda")
    Skt = torch.zeros((R.M, R.N), dtype=torch.complex64, device="cuda")
    bad_step = dataclasses.replace(ok, vc=Axis(ok.vc.start, ok.vc.step * 1.01, 3))
    bad_fold = dataclasses.replace(ok, vc=Axis(ok.vc.start + 0.3 * ok.vc.step, ok.vc.step, 3))
    for bad in (bad_step, bad_fold):
        with pytest.raises(g.GrftError):
            g.dskt_coarse_rm(R, Skt, bad, 0, 3, Z)
    with pytest.raises(g.GrftError):                     # Fv = 32: no such transform length
        g.dskt_fine_dfm_fft(R, Z, dataclasses.replace(ok, Fv=32), 0, 3, None,
                            torch.empty((96, 2, R.N), device="cuda"))
    assert g.grft_sync_status() == 0


_CHUNK_CODE = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g, synth
sc = synth.dskt_m64()
R, ds = sc.radar, sc.ds
s = synth.make_echo(R, sc.targets, sc.seed)
P = g.dsktmfp(R, torch.from_numpy(s).cuda(), ds)
assert g.grft_sync_status() == 0
np.save(sys.argv[1], P.cpu().numpy())
"""


def test_dskt_mfp_chunks_over_folding_factors(cuda_lib, tmp_path):
    """A budget of two folding-factor rows (4 chunks for q in [-3, 3]) gives the same map,
    bit for bit, as one chunk."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sc = synth.dskt_m64()
    row_bytes = sc.ds.ac.count * sc.radar.M * sc.ds.r0_count * 8
    outs = []
    for name, budget in (("one", None), ("four", 2 * row_bytes + 64)):
        env = dict(os.environ)
        env.pop("DSGRFT_SPLIT_BUDGET_BYTES", None)
        if budget:
            env["DSGRFT_SPLIT_BUDGET_BYTES"] = str(budget)
        out = str(tmp_path / (name + ".npy"))
        r = subprocess.run([sys.executable, "-c", _CHUNK_CODE % root, out], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])


def test_kt_edges_max_range_min_pulses_and_empty(cuda_lib):
    """N = 8192 (the largest range length) with M = 16 (the fewest pulses): keystone and
    coarse stage on every output; the fine stage with M = 16 zero-padded into a 64-point
    transform; an empty cell range writes nothing."""
    g = cuda_lib
    R = Radar(M=16, N=8192, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    s = synth.make_echo(R, [Target(5000.3, 150.0, 4.0, complex(2.0, -1.0))], 44)
    Skt = _keystone(g, R, s)
    ykt = oracle.keystone(R, s)
    assert rel_peak_err(Skt, ykt[:, _slots(g, R.N)]) <= TOL_FP32
    ds = synth.kt_grid(R, -1, 3, Axis(-5.0, 10.0, 2), 2, L=64, r0_begin=4990, r0_count=33)
    Z = torch.empty((ds.n_cells, R.M, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_coarse_rm(R, torch.from_numpy(Skt).cuda(), ds, 0, ds.n_cells, Z)
    assert g.grft_sync_status() == 0
    Zo = oracle.kt_coarse_rm(R, ykt, ds, 0, ds.n_cells)
    assert rel_peak_err(Z.cpu().numpy(), Zo) <= TOL_FP32
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
    g.dskt_fine_dfm_fft(R, Z, ds, 0, ds.n_cells, Y, None)
    assert g.grft_sync_status() == 0
    Yo = oracle.dskt_map(R, s, ds, ykt=ykt)
    assert rel_peak_err(Y.cpu().numpy(), Yo) <= TOL_FP32
    sentinel = torch.full_like(Z, complex(7.0, 7.0))
    g.dskt_coarse_rm(R, torch.from_numpy(Skt).cuda(), ds, 2, 0, sentinel)
    torch.cuda.synchronize()
    assert torch.all(sentinel == complex(7.0, 7.0))
