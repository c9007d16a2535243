"""Host-side logic of the multi-GPU benchmark on CPU ranks (gloo, world size 2): the
job-level timing is the slowest rank's, throughput counts every rank's units, and each
rank draws its own independent CPI.  Nothing on the data path crosses ranks."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_layout()
        t = bench.max_over_ranks(10.0 + 5.0 * rank)                 # rank 1 is slower
        sc = synth.ds_m512(run=r)
        s = synth.make_echo(sc.radar, sc.targets[:1], sc.seed)
        out.put((r, w, lr, t, float(np.abs(s[:4, :64]).sum()), sc.seed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_own_distinct_cpis():
    world, port = 2, 29641
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert [x[2] for x in res] == [0, 1]
    assert all(x[3] == 15.0 for x in res)                        # max over ranks on every rank
    assert res[0][5] != res[1][5] and res[0][4] != res[1][4]     # independent CPIs


def test_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2.0 ** 39, 1, 0.01) == pytest.approx(2.0 ** 39 / 0.01)
    assert bench.job_rate(2.0 ** 39, 4, 0.01) == pytest.approx(4 * 2.0 ** 39 / 0.01)
    assert bench.max_over_ranks(3.5) == 3.5                      # no process group: the value itself
