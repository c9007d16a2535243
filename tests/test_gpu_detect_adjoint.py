"""GPU parity of CA-CFAR + local maximum + top-K, of the trajectory adjoint (against the
FP64 oracle gradient and central differences), of the autograd.Function and of the
refinement loop, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import CFAR, Target
from tests.helpers import TOL_FP32

pytestmark = pytest.mark.gpu


def _ambiguous(P, cfar, idx_set_diff):
    """Cells whose decision is within FP32 rounding of the CFAR threshold or of a tie."""
    nv, na, nr0 = P.shape
    G, T = cfar.guard, cfar.train
    out = []
    for idx in idx_set_diff:
        vi, rem = divmod(int(idx), na * nr0)
        ai, n = divmod(rem, nr0)
        row = P[vi, ai]
        tr = [row[j] for j in list(range(n - G - T, n - G)) + list(range(n + G + 1, n + G + T + 1)) if 0 <= j < nr0]
        thr = (cfar.pfa ** (-1.0 / len(tr)) - 1.0) * sum(tr) if tr else np.inf
        nb = P[max(vi - 1, 0):vi + 2, max(ai - 1, 0):ai + 2, max(n - 1, 0):n + 2]
        close_thr = abs(row[n] - thr) <= 1e-5 * max(thr, 1e-30)
        close_nb = np.sort(nb.ravel())[-2] >= row[n] * (1 - 1e-6)
        out.append(close_thr or close_nb)
    return all(out)


@pytest.mark.parametrize("nr0", [4096, 2080, 96, 32, 3001, 2052, 1043, 50])
def test_cfar_topk_matches_oracle_on_same_power(cuda_lib, nr0):
    """Row lengths: whole 1024-bin warp chunks, multiples of 32 with a partial last chunk or
    shorter than one chunk (the tensor-map path, zero-filled past the row), ragged and
    unaligned rows, a second chunk holding a few bins, a row shorter than the training
    window.  Targets also sit on
    lane and chunk boundaries, and two equal adjacent peaks test the index tie-break."""
    g = cuda_lib
    rng = np.random.default_rng(nr0)
    nv, na = 24, 7
    P = rng.exponential(1.0, size=(nv, na, nr0)).astype(np.float32)
    for k in range(40):       # strong and weak targets
        P[rng.integers(nv), rng.integers(na), rng.integers(nr0)] = np.float32(rng.uniform(20, 200))
    for n in (0, 31, 32, 1023, 1024, 1025, nr0 - 1):
        if 0 <= n < nr0:
            P[rng.integers(nv), rng.integers(na), n] = np.float32(rng.uniform(50, 300))
    if nr0 > 8:
        P[5, 3, nr0 // 2] = P[5, 3, nr0 // 2 + 1] = np.float32(400.0)
    cfar = CFAR(2, 16, 1e-4)
    K = 64
    out, n_out = g.detect_peaks(torch.from_numpy(P).cuda(), cfar, K)
    dets, total = g.decode_detections(out, n_out, K)
    idx_o, p_o, tot_o = oracle.cfar_detect(P.astype(np.float64), cfar, K)
    gi, oi = set(dets["idx"].tolist()), set(idx_o.tolist())
    if gi != oi or total != tot_o:
        assert _ambiguous(P.astype(np.float64), cfar, (gi ^ oi))
    else:
        assert dets["idx"].tolist() == idx_o.tolist()
        np.testing.assert_array_equal(dets["p"], p_o.astype(np.float32))
    assert g.grft_sync_status() == 0


@pytest.mark.parametrize("nr0", [3001, 1043, 50, 2052, 2080])
def test_cfar_kernels_agree(cuda_lib, nr0, monkeypatch):
    """The pipelined kernels (tensor-map copies for rows of a multiple of 32 bins, 16-byte
    copies for 16-byte aligned rows, 4-byte copies for rows at any offset) and the fallback
    one-chunk-per-warp kernel (DSGRFT_CFAR_WARP) give the same detections and totals."""
    g = cuda_lib
    rng = np.random.default_rng(nr0 + 1)
    P = rng.exponential(1.0, size=(13, 5, nr0)).astype(np.float32)
    for k in range(60):
        P[rng.integers(13), rng.integers(5), rng.integers(nr0)] = np.float32(rng.uniform(15, 200))
    Pd = torch.from_numpy(P).cuda()
    cfar = CFAR(2, 16, 1e-3)
    K = 256
    a = g.decode_detections(*g.detect_peaks(Pd, cfar, K), K)
    monkeypatch.setenv("DSGRFT_CFAR_WARP", "1")
    b = g.decode_detections(*g.detect_peaks(Pd, cfar, K), K)
    assert a[1] == b[1] and a[1] > 10
    assert a[0].tobytes() == b[0].tobytes()
    assert g.grft_sync_status() == 0


def test_topk_radix_select_path_and_ties(cuda_lib):
    """More than 8192 candidates (fixed threshold, every local max passes) takes the radix
    select path; equal powers are ordered by index."""
    g = cuda_lib
    rng = np.random.default_rng(5)
    P = rng.exponential(1.0, size=(64, 16, 2048)).astype(np.float32)
    P[3, 4, 100] = P[10, 2, 900] = P[50, 9, 7] = np.float32(77.0)
    cfar = CFAR(2, 16, 1e-3, fixed_thresh=0.5, mode=1)
    K = 500
    out, n_out = g.detect_peaks(torch.from_numpy(P).cuda(), cfar, K)
    dets, total = g.decode_detections(out, n_out, K)
    idx_o, p_o, tot_o = oracle.cfar_detect(P.astype(np.float64), cfar, K)
    assert total == tot_o and total > 8192
    assert dets["idx"].tolist() == idx_o.tolist()
    assert dets["idx"][:3].tolist() == sorted(dets["idx"][:3].tolist())


def test_detection_estimates_map_to_grid_values(cuda_lib):
    g = cuda_lib
    sc = synth.plain_m64()
    s = synth.make_echo(sc.radar, sc.targets, sc.seed)
    P = g.grft(sc.radar, torch.from_numpy(s).cuda(), sc.plain)
    out, n_out = g.detect_peaks(P, CFAR(2, 16, 1e-6), 4, axes=sc.plain, dr_m=sc.radar.dr_m)
    dets, total = g.decode_detections(out, n_out, 4)
    d = dets[0]
    assert d["vi"] == 32 and d["ai"] == 8 and abs(d["n0"] - 100) <= 1
    assert d["r0_m"] == (sc.plain.r0_begin + d["n0"]) * sc.radar.dr_m
    assert abs(d["v"] - (sc.plain.v.start + d["vi"] * sc.plain.v.step)) < 1e-12
    assert abs(d["a"] - (sc.plain.a.start + d["ai"] * sc.plain.a.step)) < 1e-12


def _adj_case():
    sc = synth.ds_adjoint_m1024()
    R = sc.radar
    s = synth.make_echo(R, sc.targets, sc.seed)
    pg = sc.plain
    rng = np.random.default_rng(2)
    th = []
    for t in sc.targets[:8]:
        th.append([t.r0_bins * R.dr_m + rng.uniform(-7, 7), t.v + rng.uniform(-1, 1) * pg.v.step,
                   t.a + rng.uniform(-1, 1) * pg.a.step])
    for _ in range(8):   # noise-only points
        th.append([rng.uniform(500, 3500) * R.dr_m, rng.uniform(-290, 290), rng.uniform(-19, 19)])
    return R, s, np.array(th), pg


@pytest.mark.parametrize("gather", [0, 1])
def test_adjoint_matches_oracle_gradient(cuda_lib, gather):
    g = cuda_lib
    R, s, th, pg = _adj_case()
    es = torch.from_numpy(s).cuda()
    tht = torch.from_numpy(th).cuda()
    K = th.shape[0]
    P = torch.empty(K, device="cuda")
    Y = torch.empty(K, dtype=torch.complex64, device="cuda")
    gt = torch.empty((K, 3), dtype=torch.float64, device="cuda")
    g.dsgrft_backward(R, es, tht, gather, P=P, Y=Y, grad_theta=gt)
    Po, Yo, go = oracle.trajectory_grad(R, s, th, gather)
    assert np.abs(P.cpu().numpy() - Po).max() <= 1e-4 * Po.max()
    assert np.abs(Y.cpu().numpy() - Yo).max() <= TOL_FP32 * 10 * np.abs(Yo).max()
    gg = gt.cpu().numpy()
    k4 = 4 * np.pi / R.wavelength
    for j in range(3):
        scale = np.abs(go[:, j]).max()
        if gather == 0 and j == 0:
            # nearest gather: dP/dr0 = 2 Re(conj(Y) j k4 Y) = 0 exactly; the FP32 sums leave
            # rounding of the size of the terms 2 k4 |Y|^2 they cancel
            scale = 2 * k4 * Po.max()
        assert np.abs(gg[:, j] - go[:, j]).max() <= 1e-4 * scale, (j, np.abs(gg[:, j] - go[:, j]).max() / scale)


def test_adjoint_central_differences(cuda_lib):
    """dP/dtheta of the GPU adjoint against central differences (h = 1e-3 cell, Richardson
    extrapolated with h/2) of the FP64 forward, linear gather, at points where no gathered
    bin is crossed: 1e-4 relative."""
    g = cuda_lib
    R, s, th, pg = _adj_case()
    es = torch.from_numpy(s).cuda()
    cell = np.array([R.dr_m, pg.v.step, pg.a.step])
    K = th.shape[0]
    gt = torch.empty((K, 3), dtype=torch.float64, device="cuda")
    g.dsgrft_backward(R, es, torch.from_numpy(th).cuda(), 1, grad_theta=gt)
    gg = gt.cpu().numpy()
    # the forward in FP32 cannot resolve h = 1e-3 cell differences to 1e-4: differentiate the
    # FP64 oracle's forward instead and compare the GPU adjoint with it.  The central
    # difference at h = 1e-3 cell has a truncation error of up to about 1e-4 of the gradient
    # (the phase turns by about 0.02 rad per step across the CPI), so the h and h/2
    # differences are combined by Richardson extrapolation, (4 D(h/2) - D(h)) / 3, whose error
    # is of fourth order in h
    t = np.arange(R.M) / R.prf_hz
    ok, worst = 0, 0.0

    def cdiff(k, j, h):
        tp, tm = th[k].copy(), th[k].copy()
        tp[j] += h
        tm[j] -= h
        Pp = oracle.trajectory_grad(R, s, tp[None], 1)[0][0]
        Pm = oracle.trajectory_grad(R, s, tm[None], 1)[0][0]
        return (Pp - Pm) / (2 * h)

    for k in range(K):
        for j in range(3):
            h = 1e-3 * cell[j]
            tp, tm = th[k].copy(), th[k].copy()
            tp[j] += h
            tm[j] -= h
            xp = (tp[0] + tp[1] * t + 0.5 * tp[2] * t * t) / R.dr_m
            xm = (tm[0] + tm[1] * t + 0.5 * tm[2] * t * t) / R.dr_m
            if np.any(np.floor(xp) != np.floor(xm)):
                continue
            fd = (4.0 * cdiff(k, j, 0.5 * h) - cdiff(k, j, h)) / 3.0
            # 1e-4 relative; a gradient component within 1e-3 of its column's largest (near a
            # peak, where the relative error of any finite-precision sum grows without bound)
            # is compared at 1e-4 of that floor
            scale = max(abs(fd), 1e-3 * np.abs(gg[:, j]).max())
            worst = max(worst, abs(gg[k, j] - fd) / scale)
            assert abs(gg[k, j] - fd) <= 1e-4 * scale, (k, j, gg[k, j], fd)
            ok += 1
    print("adjoint vs central differences of the FP64 forward: worst relative error", worst, "over", ok)
    assert ok >= K


def test_grad_s_matches_oracle_and_autograd(cuda_lib):
    g = cuda_lib
    R, s, th, pg = _adj_case()
    es = torch.from_numpy(s).cuda()
    gP = np.linspace(0.5, 1.5, th.shape[0])
    gs = torch.zeros_like(es)
    g.dsgrft_backward(R, es, torch.from_numpy(th).cuda(), 1,
                      grad_P=torch.tensor(gP, dtype=torch.float32, device="cuda"), grad_s=gs)
    _, _, _, gso = oracle.trajectory_grad(R, s, th, 1, gP=gP, want_grad_s=True)
    assert np.abs(gs.cpu().numpy() - gso).max() <= 1e-4 * np.abs(gso).max()
    # the autograd.Function gives the same gradients
    e = es.clone().requires_grad_(True)
    tt = torch.from_numpy(th).cuda().requires_grad_(True)
    P = g.TrajectoryPower.apply(e, tt, R, 1)
    (P * torch.tensor(gP, dtype=torch.float32, device="cuda")).sum().backward()
    assert torch.allclose(e.grad, gs, rtol=0, atol=1e-5 * gs.abs().max().item())
    assert tt.grad.shape == (th.shape[0], 3)


def test_refine_matches_oracle(cuda_lib):
    g = cuda_lib
    sc = synth.ds_adjoint_m1024()
    R, pg = sc.radar, sc.plain
    s = synth.make_echo(R, sc.targets, sc.seed, noise=False)
    th0 = []
    for t in sc.targets:
        th0.append([round(t.r0_bins) * R.dr_m, pg.v.start + round((t.v - pg.v.start) / pg.v.step) * pg.v.step,
                    pg.a.start + round((t.a - pg.a.start) / pg.a.step) * pg.a.step])
    th0 = np.array(th0)
    cell = [R.dr_m, pg.v.step, pg.a.step]
    tht = torch.from_numpy(th0).cuda()
    Pg = torch.empty(th0.shape[0], device="cuda")
    g.dsgrft_refine(R, torch.from_numpy(s).cuda(), tht, cell, 20, 1, Pg)
    tho, Po = oracle.refine(R, s, th0, cell, 20, mode=1)
    P0 = oracle.trajectory_grad(R, s, th0, 1)[0]
    Pg = Pg.cpu().numpy()
    assert np.all(Pg >= P0 * (1 - 1e-5))
    # every target: same final power and same point to 0.05 cell
    rel = np.abs(Pg - Po) / Po
    d = np.abs(tht.cpu().numpy() - tho) / np.array(cell)
    print("refinement vs oracle: worst power difference", rel.max(), "worst distance (cells)", d.max())
    assert np.all(rel <= 1e-3), rel
    assert np.all(d.max(axis=1) <= 0.05), d
