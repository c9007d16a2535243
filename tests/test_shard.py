"""Host logic of one CPI's search split over several GPUs (paper_2403_06788_gb300.shard), run
on CPU ranks (gloo, world size 2 and 3): the coarse-v partition covers the grid once, the
halo exchange hands each rank its neighbours' border rows, and the detection lists gathered
from the ranks merge into exactly the whole map's top K (ties by index), the totals summing
to the whole map's.  Each rank's own detection uses the FP64 oracle's detector on its rows
plus halos (the GPU detector's slab scan is checked against the whole map in
test_gpu_stream_detect.py, the device merge in test_gpu_shard.py)."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NVC, FV, NA, NR0, K = 7, 4, 6, 300, 64


def _map():
    rng = np.random.default_rng(42)
    P = rng.exponential(1.0, size=(NVC * FV, NA, NR0))
    for _ in range(80):
        P[rng.integers(NVC * FV), rng.integers(NA), rng.integers(NR0)] = rng.uniform(20, 200)
    for v in range(FV - 1, NVC * FV, FV):           # peaks on every coarse-row border
        P[v, 2, 40 + v] = 150.0 + v
        P[v + 1 if v + 1 < NVC * FV else v, 3, 41 + v] = 149.0 + v
    P[FV - 1, 4, 100] = P[FV, 4, 100] = 500.0       # an equal pair across a border: index tie-break
    return P


def _sort_records(rec):
    order = np.lexsort((rec["idx"], -rec["p"].astype(np.float64)))
    return rec[order]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    import synth
    from paper_2403_06788_gb300 import DET_DTYPE, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cf = synth.CFAR(2, 16, 1e-3)
        P = _map()
        i0, i1 = shard.coarse_rows(NVC, world, rank)
        rows = (i1 - i0) * FV
        ext = torch.zeros((rows + 2, NA, NR0), dtype=torch.float64)
        ext[1:rows + 1] = torch.from_numpy(P[i0 * FV:i1 * FV])       # this rank's rows only
        shard.exchange_halos(ext[1], ext[rows], ext[0], ext[rows + 1])
        lo = 1 if rank == 0 else 0
        hi = rows + 2 if rank + 1 < world else rows + 1
        slab = ext[lo:hi].numpy()
        halo_ok = (rank == 0 or np.array_equal(ext[0].numpy(), P[i0 * FV - 1])) and \
            (rank + 1 == world or np.array_equal(ext[rows + 1].numpy(), P[i1 * FV]))
        # this rank's detections: rows of the slab outside the halo, whole-map indices
        idx, p, _ = oracle.cfar_detect(slab, cf, 1 << 16)
        v = idx // (NA * NR0)
        keep = (v >= 1 - lo) & (v < 1 - lo + rows)
        gidx = idx[keep] + (i0 * FV - (1 - lo)) * NA * NR0
        rec = np.zeros(K, dtype=DET_DTYPE)
        loc = _sort_records(np.array(list(zip(gidx, p[keep])), dtype=[("idx", "<i8"), ("p", "<f4")]))[:K]
        rec["idx"][:len(loc)] = loc["idx"]
        rec["p"][:len(loc)] = loc["p"]
        out = torch.from_numpy(rec.view(np.uint8).copy())
        n_out = torch.tensor([int(keep.sum())], dtype=torch.int32)
        lists, totals = shard.gather_detections(out, n_out)
        # the merge of the gathered lists (the device kernel's rule, on the host)
        allrec = lists.numpy().view(DET_DTYPE).reshape(world, K)
        tot = totals.numpy()
        merged = _sort_records(np.concatenate([allrec[r][:min(K, tot[r])] for r in range(world)]))[:K]
        q.put((rank, (i0, i1), bool(halo_ok), merged["idx"].tolist(), merged["p"].tolist(), int(tot.sum())))
    finally:
        dist.destroy_process_group()


def test_coarse_rows_partition():
    sys.path.insert(0, ROOT)
    from paper_2403_06788_gb300 import shard
    for nvc in (1, 7, 32):
        for world in range(1, min(nvc, 9) + 1):
            parts = [shard.coarse_rows(nvc, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == nvc
            assert all(a[1] == b[0] for a, b in zip(parts[:-1], parts[1:]))
            sizes = [b - a for a, b in parts]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.coarse_rows(4, 5, 0)


@pytest.mark.parametrize("world,port", [(2, 29651), (3, 29653)])
def test_sharded_detection_merges_to_whole_map_topk(world, port):
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    idx_o, p_o, tot_o = oracle.cfar_detect(_map(), synth.CFAR(2, 16, 1e-3), K)
    assert tot_o > K                                   # the top K is a real selection
    for rank, part, halo_ok, idx, pw, tot in res:
        assert halo_ok, rank
        assert idx == idx_o.tolist(), rank             # same cells, same order, on every rank
        assert np.array_equal(np.float32(pw), np.float32(p_o))
        assert tot == tot_o
    assert res[0][1][0] == 0 and res[-1][1][1] == NVC
