"""GPU checks at the sizes of the precision configuration (M=2048 x N=8192, fine 256 x 64:
3.4e10 hypotheses, run here one coarse-v slab at a time) and of the differentiation
configuration (M=1024 x N=4096, DS forward, top-1000 CFAR detections, adjoint and 20
refinement steps), against the FP64 oracle on sampled outputs."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.wrap import ds_rows_of_canonical
from tests.helpers import TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu


def test_precision_config_slab_bf16x3_and_fp16x3(cuda_lib):
    g = cuda_lib
    sc = synth.ds_precision_m2048()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets, sc.seed)
    echo = torch.from_numpy(s).cuda()
    pg = ds.plain_equivalent()
    # the coarse-v row holding the strongest target
    t = max(sc.targets, key=lambda t: abs(t.amp))
    i_row = min(int((t.v - pg.v.start) // ds.vc.step), ds.vc.count - 1)
    cb, cc = i_row * ds.ac.count, ds.ac.count
    nv, na = ds.Fv, ds.ac.count * ds.Fa
    rng = np.random.default_rng(0)
    vloc = list(rng.integers(0, nv, 10))
    af = list(rng.integers(0, na, 10))
    jt = int(round((t.v - pg.v.start) / pg.v.step)) - i_row * ds.Fv
    kt = int(round((t.a - pg.a.start) / pg.a.step))
    vloc.append(int(np.clip(jt, 0, nv - 1)))
    af.append(int(np.clip(kt, 0, na - 1)))
    cell, fine = ds_rows_of_canonical(ds, np.array(vloc) + i_row * ds.Fv, np.array(af))
    Yo = oracle.dsgrft_rows(R, s, ds, cell, fine)
    errs = {}
    for prec in ("bf16x3", "fp16x3", "fp16x2", "fp16x1"):
        Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
        g.dsgrft_fine_dfm(R, None, echo, ds, cb, cc, prec, Y, None)
        assert g.grft_sync_status() == 0
        Yg = Y[torch.as_tensor(vloc, device="cuda"), torch.as_tensor(af, device="cuda")].cpu().numpy()
        errs[prec] = rel_peak_err(Yg, Yo)
        del Y
        torch.cuda.empty_cache()
    print("precision config max rel peak error:", errs)
    for prec, e in errs.items():
        assert e <= TOL_SPLIT, (prec, e)


def test_differentiation_config_pipeline(cuda_lib):
    """DS forward (bf16x3) -> CA-CFAR top-1000 -> 20 ascent steps with the adjoint (linear
    gather).  Refined powers and points of each of 32 detections agree with the FP64
    oracle's refinement; gradients agree with the oracle's to 1e-4 of scale."""
    g = cuda_lib
    sc = synth.ds_adjoint_m1024()
    R, ds = sc.radar, sc.ds
    pg = ds.plain_equivalent()
    s = synth.make_echo(R, sc.targets, sc.seed)
    echo = torch.from_numpy(s).cuda()
    P = g.dsgrft(R, echo, ds, precision="bf16x3")
    out, n_out = g.detect_peaks(P, synth.CFAR(2, 16, 1e-6), 1000, axes=pg, dr_m=R.dr_m)
    dets, total = g.decode_detections(out, n_out, 1000)
    del P
    assert dets.size >= 16
    th0 = np.stack([dets["r0_m"], dets["v"], dets["a"]], axis=1).astype(np.float64)
    cell = [R.dr_m, pg.v.step, pg.a.step]
    tht = torch.from_numpy(th0.copy()).cuda()
    Pr = torch.empty(th0.shape[0], device="cuda")
    g.dsgrft_refine(R, echo, tht, cell, 20, 1, Pr)
    P0 = torch.empty(th0.shape[0], device="cuda")
    g.dsgrft_backward(R, echo, torch.from_numpy(th0).cuda(), 1, P=P0)
    assert g.grft_sync_status() == 0
    assert torch.all(Pr >= P0 * (1 - 1e-5))
    sel = np.arange(min(32, th0.shape[0]))
    tho, Po = oracle.refine(R, s, th0[sel], cell, 20, mode=1)
    Pg = Pr.cpu().numpy()[sel]
    rel = np.abs(Pg - Po) / Po
    d = np.abs(tht.cpu().numpy()[sel] - tho) / np.array(cell)
    print("config-5 refinement vs oracle: worst power difference", rel.max(), "worst distance (cells)", d.max())
    assert np.all(rel <= 1e-3), rel
    assert np.all(d.max(axis=1) <= 0.05), d
    # adjoint at the on-grid starting points (off the sub-grid peak, so the gradient is
    # well away from zero) against the FP64 gradient
    thr = th0[sel]
    gt = torch.empty((sel.size, 3), dtype=torch.float64, device="cuda")
    g.dsgrft_backward(R, echo, torch.from_numpy(thr).cuda(), 1, grad_theta=gt)
    _, _, go = oracle.trajectory_grad(R, s, thr, 1)
    gg = gt.cpu().numpy()
    for j in range(3):
        scale = np.abs(go[:, j]).max()
        assert np.abs(gg[:, j] - go[:, j]).max() <= 1e-4 * max(scale, 1e-30) + 1e-6 * scale
