"""GPU: DS-GRFT with the acceleration rate (P = 3, dsgrft3_fine_dfm) through the C ABI
against the FP64 numpy oracle (oracle/p3.py): every output of a small case with ragged
tiles on every axis, the trivial b axis equal to the P = 2 path bit for bit, a cell
sub-range written into its v-slab only, sampled rows and target focus on the
2.1e9-hypothesis ds3_m512 grid, an empty cell range, and the rejection of FP32."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import Axis, DSGrid, DSGrid3, Radar, Target
from tests.helpers import TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu


def _small():
    R = Radar(M=100, N=400, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    g3 = DSGrid3(17, 300, Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 2), Axis(-30.0, 40.0, 3), 8, 4, 3)
    tg = [Target(17 + 120.0, -21.0, 1.2, complex(3.0, -1.0), 35.0),
          Target(17 + 251.3, 3.0, -2.0, complex(1.0, 2.0), -20.0)]
    return R, g3, synth.make_echo(R, tg, 13)


def _rows(g3):
    nv, na, nb = g3.vc.count * g3.Fv, g3.ac.count * g3.Fa, g3.bc.count * g3.Fb
    vi, ai, bi = np.meshgrid(np.arange(nv), np.arange(na), np.arange(nb), indexing="ij")
    i, k = np.divmod(vi.ravel(), g3.Fv)
    l, q = np.divmod(ai.ravel(), g3.Fa)
    w, u = np.divmod(bi.ravel(), g3.Fb)
    cell = (i * g3.ac.count + l) * g3.bc.count + w
    fine = (k * g3.Fa + q) * g3.Fb + u
    return cell, fine, (nv, na, nb)


@pytest.mark.parametrize("precision,guard", [("bf16x3", 1e-4), ("fp16x3", 1e-4), ("fp16x2", 5e-4), ("fp16x1", 5e-4)])
def test_p3_every_output_small(cuda_lib, precision, guard):
    g = cuda_lib
    R, g3, s = _small()
    P, Y = g.dsgrft3(R, torch.from_numpy(s).cuda(), g3, precision=precision, want_Y=True)
    assert g.grft_sync_status() == 0
    cell, fine, shape = _rows(g3)
    Yo = oracle.dsgrft3_rows(R, s, g3, cell, fine).reshape(*shape, g3.r0_count)
    err = rel_peak_err(Y.cpu().numpy(), Yo)
    assert err <= TOL_SPLIT and err <= guard, err
    assert rel_peak_err(P.cpu().numpy(), np.abs(Yo) ** 2) <= 2 * TOL_SPLIT


def test_p3_trivial_b_axis_is_the_p2_path(cuda_lib):
    """One b cell at 0 and one fine b offset (0): the P = 3 launch computes exactly the P = 2
    bins, phases and dechirp values, so its output equals dsgrft_fine_dfm bit for bit."""
    g = cuda_lib
    R, g3, s = _small()
    g3 = dataclasses.replace(g3, bc=Axis(0.0, 0.0, 1), Fb=1)
    ds = DSGrid(g3.r0_begin, g3.r0_count, g3.vc, g3.ac, g3.Fv, g3.Fa)
    es = torch.from_numpy(s).cuda()
    Y3 = g.dsgrft3(R, es, g3, precision="bf16x3", want_Y=True, want_P=False)
    Y2 = g.dsgrft(R, es, ds, precision="bf16x3", want_Y=True, want_P=False)
    assert torch.equal(Y3[:, :, 0, :], Y2)


def test_p3_cell_subrange_writes_its_slab(cuda_lib):
    g = cuda_lib
    R, g3, s = _small()
    es = torch.from_numpy(s).cuda()
    per_row = g3.ac.count * g3.bc.count
    cb, cc = per_row + 2, 3                    # row i = 1, cells (l, w) = (0, 2), (1, 0), (1, 1)
    shape = (g3.Fv, g3.ac.count * g3.Fa, g3.bc.count * g3.Fb, g3.r0_count)
    Y = torch.full(shape, complex(-1.0, 0.0), dtype=torch.complex64, device="cuda")
    g.dsgrft3_fine_dfm(R, es, g3, cb, cc, "bf16x3", Y, None)
    assert g.grft_sync_status() == 0
    Yn = Y.cpu().numpy()
    for c in range(cb, cb + cc):
        l, w = divmod(c - per_row, g3.bc.count)
        fine = np.arange(g3.Fv * g3.Fa * g3.Fb)
        Yo = oracle.dsgrft3_rows(R, s, g3, np.full(fine.size, c), fine).reshape(g3.Fv, g3.Fa, g3.Fb, g3.r0_count)
        got = Yn[:, l * g3.Fa:(l + 1) * g3.Fa, w * g3.Fb:(w + 1) * g3.Fb]
        assert rel_peak_err(got, Yo) <= TOL_SPLIT
    # the first cell of the row, (l, w) = (0, 0), is outside the range and untouched
    assert np.all(Yn[:, 0:g3.Fa, 0:g3.Fb] == complex(-1.0, 0.0))


def test_p3_m512_sampled_rows_and_focus(cuda_lib):
    g = cuda_lib
    sc = synth.ds3_m512()
    R, g3 = sc.radar, sc.ds3
    s = synth.make_echo(R, sc.targets, sc.seed)
    P, = [g.dsgrft3(R, torch.from_numpy(s).cuda(), g3, precision="bf16x3")]
    assert g.grft_sync_status() == 0
    assert P.shape == (8 * 64, 8 * 8, 4 * 4, 4096)
    vstart = g3.vc.start - 0.5 * g3.vc.step
    astart = g3.ac.start - 0.5 * g3.ac.step
    bstart = g3.bc.start - 0.5 * g3.bc.step
    dv, da, db = g3.vc.step / g3.Fv, g3.ac.step / g3.Fa, g3.bc.step / g3.Fb
    for t in sc.targets:
        iv, ia, ib = (int(round((t.v - vstart) / dv)), int(round((t.a - astart) / da)),
                      int(round((t.b - bstart) / db)))
        ir = int(round(t.r0_bins))
        box = P[max(iv - 2, 0):iv + 3, max(ia - 2, 0):ia + 3, max(ib - 1, 0):ib + 2, max(ir - 1, 0):ir + 2]
        assert float(box.max()) >= 0.2 * (abs(t.amp) * R.M) ** 2, t
    # sampled rows (every r0) against the oracle, including the strongest target's row
    t = max(sc.targets, key=lambda t: abs(t.amp))
    rng = np.random.default_rng(3)
    vi = list(rng.integers(0, P.shape[0], 5)) + [int(round((t.v - vstart) / dv))]
    ai = list(rng.integers(0, P.shape[1], 5)) + [int(round((t.a - astart) / da))]
    bi = list(rng.integers(0, P.shape[2], 5)) + [int(round((t.b - bstart) / db))]
    i, k = np.divmod(np.asarray(vi), g3.Fv)
    l, q = np.divmod(np.asarray(ai), g3.Fa)
    w, u = np.divmod(np.asarray(bi), g3.Fb)
    cell = (i * g3.ac.count + l) * g3.bc.count + w
    fine = (k * g3.Fa + q) * g3.Fb + u
    del P
    torch.cuda.empty_cache()
    Y = g.dsgrft3(R, torch.from_numpy(s).cuda(), g3, precision="bf16x3", want_Y=True, want_P=False)
    Yg = Y[torch.as_tensor(vi, device="cuda"), torch.as_tensor(ai, device="cuda"),
           torch.as_tensor(bi, device="cuda")].cpu().numpy()
    del Y
    torch.cuda.empty_cache()
    Yo = oracle.dsgrft3_rows(R, s, g3, cell, fine)
    assert rel_peak_err(Yg, Yo) <= TOL_SPLIT


def test_p3_rejects_fp32(cuda_lib):
    g = cuda_lib
    R, g3, s = _small()
    with pytest.raises(g.GrftError):
        g.dsgrft3(R, torch.from_numpy(s).cuda(), g3, precision="fp32")
    assert g.grft_sync_status() == 0


def test_p3_empty_cell_range_writes_nothing(cuda_lib):
    g = cuda_lib
    R, g3, s = _small()
    shape = (g3.vc.count * g3.Fv, g3.ac.count * g3.Fa, g3.bc.count * g3.Fb, g3.r0_count)
    P = torch.full(shape, 3.0, device="cuda")
    g.dsgrft3_fine_dfm(R, torch.from_numpy(s).cuda(), g3, 5, 0, "bf16x3", None, P)
    torch.cuda.synchronize()
    assert g.grft_sync_status() == 0 and torch.all(P == 3.0)


P3_CODE = r"""
import sys, dataclasses, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g
from tests.test_gpu_p3 import _small
R, g3, s = _small()
g3 = dataclasses.replace(g3, Fb=int(sys.argv[2]))
P, Y = g.dsgrft3(R, torch.from_numpy(s).cuda(), g3, precision=sys.argv[3], want_Y=True)
assert g.grft_sync_status() == 0
np.save(sys.argv[1], Y.cpu().numpy())
"""


@pytest.mark.parametrize("Fb,precision", [(3, "fp16x2"), (4, "bf16x3"), (2, "fp16x1")])
def test_p3_pair_form_matches_4m_form_and_oracle(cuda_lib, tmp_path, Fb, precision):
    """Mirrored hypotheses on all three fine axes ((k, q, u) and (Fv - k, Fa - q, Fb - u)
    have conjugate dechirp rows; pair_slot3): the pair form of the P = 3 contraction matches
    the 4M form (DSGRFT_PAIR=0) within the split tolerance and the FP64 oracle on every
    output, for odd and even rate-offset counts."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def run(name, **env):
        out = os.path.join(str(tmp_path), name + ".npy")
        e = dict(os.environ)
        e.update(env)
        r = subprocess.run([sys.executable, "-c", P3_CODE % root, out, str(Fb), precision], env=e,
                           capture_output=True, text=True, timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        return np.load(out)

    Yp = run("pair")
    Y4 = run("m4", DSGRFT_PAIR="0")
    R, g3, s = _small()
    g3 = dataclasses.replace(g3, Fb=Fb)
    cell, fine, shape = _rows(g3)
    Yo = oracle.dsgrft3_rows(R, s, g3, cell, fine).reshape(*shape, g3.r0_count)
    ep, e4 = rel_peak_err(Yp, Yo), rel_peak_err(Y4, Yo)
    print(f"P=3 Fb={Fb} {precision}: pair form {ep:.3g}, 4M form {e4:.3g} of peak")
    assert ep <= TOL_SPLIT and e4 <= TOL_SPLIT
    assert ep <= 2 * e4 + 1e-6
    assert rel_peak_err(Yp, Y4) <= TOL_SPLIT
