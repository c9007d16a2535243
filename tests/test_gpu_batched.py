"""GPU: many CPIs of uneven pulse and range-bin counts in one batched call (persistent
tensor-core launches), checked against each CPI's standalone call (bit-identical: same
tables, same contraction order) and against the FP64 oracle on sampled rows; graph
capture and replay; the chunked (multi-round) split operand."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.wrap import ds_rows_of_canonical
from synth import Axis, DSGrid, Radar, Target
from tests.helpers import TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _grid():
    return DSGrid(0, 1, Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 2), 16, 8)


def _items(shapes, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i, (M, N, r0b, r0c) in enumerate(shapes):
        R = Radar(M=M, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
        tg = [Target(float(rng.uniform(r0b + 20, r0b + r0c - 20)), float(rng.uniform(-40, 10)),
                     float(rng.uniform(-4, 4)), complex(2.0, 1.0))]
        out.append((R, r0b, r0c, synth.make_echo(R, tg, 100 + i)))
    return out


def _run_batch(g, grid, items, precision="bf16x3", want_Y=False):
    nv, na = grid.vc.count * grid.Fv, grid.ac.count * grid.Fa
    batch, outs = [], []
    for R, r0b, r0c, s in items:
        e = torch.from_numpy(s).cuda()
        P = torch.full((nv, na, r0c), -1.0, device="cuda")
        Y = torch.zeros((nv, na, r0c), dtype=torch.complex64, device="cuda") if want_Y else None
        batch.append({"echo": e, "P": P, "Y": Y, "r0_begin": r0b, "r0_count": r0c})
        outs.append((P, Y))
    g.dsgrft_fine_dfm_batched(items[0][0], grid, batch, precision)
    return batch, outs


def _standalone(g, R, s, grid, r0b, r0c, precision="bf16x3"):
    import dataclasses
    gi = dataclasses.replace(grid, r0_begin=r0b, r0_count=r0c)
    return g.dsgrft(R, torch.from_numpy(s).cuda(), gi, precision=precision, want_Y=True)


SHAPES = [(100, 500, 0, 500), (256, 1200, 37, 1000), (333, 777, 100, 300), (64, 256, 0, 256),
          (1024, 2048, 512, 1024)]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3", "fp16x2", "fp16x1"])
def test_batched_equals_standalone_and_oracle(cuda_lib, precision):
    g = cuda_lib
    grid = _grid()
    items = _items(SHAPES)
    batch, outs = _run_batch(g, grid, items, precision, want_Y=True)
    assert g.grft_sync_status() == 0
    rng = np.random.default_rng(1)
    for (R, r0b, r0c, s), (P, Y) in zip(items, outs):
        Ps, Ys = _standalone(g, R, s, grid, r0b, r0c, precision)
        assert torch.equal(P, Ps) and torch.equal(Y, Ys)
        import dataclasses
        gi = dataclasses.replace(grid, r0_begin=r0b, r0_count=r0c)
        vf = rng.integers(0, grid.vc.count * grid.Fv, 6)
        af = rng.integers(0, grid.ac.count * grid.Fa, 6)
        cell, fine = ds_rows_of_canonical(gi, vf, af)
        Yo = oracle.dsgrft_rows(R, s, gi, cell, fine)
        Yg = Y[torch.as_tensor(vf, device="cuda"), torch.as_tensor(af, device="cuda")].cpu().numpy()
        assert rel_peak_err(Yg, Yo) <= TOL_SPLIT


def test_batched_more_items_than_one_launch_holds(cuda_lib):
    """70 CPIs (> 64 items per launch) run in two rounds; every CPI equals its standalone run."""
    g = cuda_lib
    grid = DSGrid(0, 1, Axis(-40.0, 18.75, 2), Axis(-2.5, 5.0, 1), 8, 4)
    rng = np.random.default_rng(3)
    shapes = [(int(rng.integers(16, 96)), int(rng.integers(130, 400)), 0, 0) for _ in range(70)]
    shapes = [(M, N, 0, N) for (M, N, _, _) in shapes]
    items = _items(shapes, seed=5)
    batch, outs = _run_batch(g, grid, items)
    for (R, r0b, r0c, s), (P, _) in zip(items, outs):
        Ps, _ = _standalone(g, R, s, grid, r0b, r0c)
        assert torch.equal(P, Ps)


def test_batched_graph_capture_and_replay(cuda_lib):
    g = cuda_lib
    grid = _grid()
    items = _items(SHAPES[:3])
    batch, outs = _run_batch(g, grid, items)        # first call sizes the workspace
    ref = [P.clone() for P, _ in outs]
    for P, _ in outs:
        P.fill_(-1.0)
    R0 = items[0][0]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        g.dsgrft_fine_dfm_batched(R0, grid, batch, "bf16x3")
    for _ in range(2):
        for P, _ in outs:
            P.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        for (P, _), r in zip(outs, ref):
            assert torch.equal(P, r)


def test_split_operand_in_several_rounds_matches_one_round(cuda_lib, tmp_path):
    """A small split-operand budget (environment override, read once per process) makes the
    DS call run one cell per round, split and contraction pipelined over two buffers on two
    streams; the output matches the oracle, equals the single-round run bit for bit, and a
    captured graph of the pipelined call replays to the same values."""
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import paper_2403_06788_gb300 as g, synth, oracle
from synth import Axis, DSGrid, Radar, Target
R = Radar(M=200, N=900, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
ds = DSGrid(3, 700, Axis(-40.0, 18.75, 3), Axis(-2.5, 5.0, 3), 16, 8)
s = synth.make_echo(R, [Target(300.0, -20.0, 1.0, complex(3.0, 0.0))], 9)
echo = torch.from_numpy(s).cuda()
Yt = g.dsgrft(R, echo, ds, precision="bf16x3", want_Y=True, want_P=False)
Y = Yt.cpu().numpy()
Yo = oracle.dsgrft_full(R, s, ds)
err = np.abs(Y - Yo).max() / np.abs(Yo).max()
assert g.grft_sync_status() == 0
np.save(sys.argv[1], Y)
nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
Yc = torch.zeros((nv, na, ds.r0_count), dtype=torch.complex64, device="cuda")
st = torch.cuda.Stream()
torch.cuda.synchronize()
graph = torch.cuda.CUDAGraph()
with torch.cuda.graph(graph, stream=st):
    g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.vc.count * ds.ac.count, "bf16x3", Yc, None)
for _ in range(2):
    Yc.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(Yc, Yt)
assert g.grft_sync_status() == 0
print("ERR", err)
""" % ROOT
    outs = []
    for rounds_env in ({"DSGRFT_SPLIT_BUDGET_BYTES": str(4 * 768 * 448 * 2)},   # one cell per round
                       {"DSGRFT_ROUNDS": "1"}):
        env = dict(os.environ, **rounds_env)
        path = os.path.join(str(tmp_path), "Y%d.npy" % len(outs))
        r = subprocess.run([sys.executable, "-c", code, path], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        err = float(r.stdout.split("ERR")[1])
        assert err <= 1e-4
        outs.append(np.load(path))
    assert np.array_equal(outs[0], outs[1])


def test_ds_batch_shaped_batch_sampled(cuda_lib):
    """Eight CPIs drawn as in the batching configuration (M in [256, 2048], N in [1024, 8192],
    1-16 targets, coarse 32 x 8 cells, fine 64 x 16), full grids, sampled rows vs the oracle."""
    g = cuda_lib
    cpis = synth.ds_batch(n_cpi=8)
    grid = cpis[0].ds
    nv, na = grid.vc.count * grid.Fv, grid.ac.count * grid.Fa
    batch, data = [], []
    for sc in cpis:
        s = synth.make_echo(sc.radar, sc.targets, sc.seed)
        P = torch.empty((nv, na, sc.radar.N), device="cuda")
        batch.append({"echo": torch.from_numpy(s).cuda(), "P": P, "Y": None, "r0_begin": 0,
                      "r0_count": sc.radar.N})
        data.append((sc, s, P))
    g.dsgrft_fine_dfm_batched(cpis[0].radar, grid, batch, "bf16x3")
    assert g.grft_sync_status() == 0
    rng = np.random.default_rng(4)
    for sc, s, P in data:
        import dataclasses
        gi = dataclasses.replace(grid, r0_count=sc.radar.N)
        pg = gi.plain_equivalent()
        vf = list(rng.integers(0, nv, 2)) + [int(round((t.v - pg.v.start) / pg.v.step)) for t in sc.targets[:1]]
        af = list(rng.integers(0, na, 2)) + [int(round((t.a - pg.a.start) / pg.a.step)) for t in sc.targets[:1]]
        vf, af = np.clip(vf, 0, nv - 1), np.clip(af, 0, na - 1)
        cell, fine = ds_rows_of_canonical(gi, vf, af)
        Po = np.abs(oracle.dsgrft_rows(sc.radar, s, gi, cell, fine)) ** 2
        Pg = P[torch.as_tensor(vf, device="cuda"), torch.as_tensor(af, device="cuda")].cpu().numpy()
        assert rel_peak_err(Pg, Po) <= 2 * TOL_SPLIT
        del P
