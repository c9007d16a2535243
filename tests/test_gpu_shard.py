"""GPU: the device side of one CPI's search split over several GPUs, emulated on one GPU one
part after the other (no part waits on another).  The DS map's coarse-v rows are cut into
the blocks shard.coarse_rows gives each rank; each block is scanned with its neighbours'
border rows as halos and keeps its top K (detect_peaks_begin / add / end, as each rank
does); detect_merge of the lists, gathered into one buffer as the all-gather leaves them,
equals detect_peaks over the whole map (records, order and total)."""
import numpy as np
import pytest
import torch

import synth
from paper_2403_06788_gb300 import shard
from synth import CFAR, Axis, DSGrid, Radar, Target

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 5])
def test_sharded_lists_merge_to_whole_map(cuda_lib, world):
    g = cuda_lib
    R = Radar(M=100, N=700, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(17, 300, Axis(-40.0, 18.75, 5), Axis(-2.5, 5.0, 3), 8, 8)
    s = synth.make_echo(R, [Target(137.0, -21.0, 1.2, complex(3.0, -1.0)),
                            Target(268.3, 3.0, -2.0, complex(1.0, 2.0))], 3)
    echo = torch.from_numpy(s).cuda()
    pg = ds.plain_equivalent()
    cf = CFAR(2, 16, 1e-2)
    K = 128
    P = g.dsgrft(R, echo, ds, precision="fp16x2")
    whole = g.detect_peaks(P, cf, K, axes=pg, dr_m=R.dr_m)
    nvc, Fv = ds.vc.count, ds.Fv
    na, nr0 = int(P.shape[1]), int(P.shape[2])
    lists = torch.zeros((world, K * g._abi.DET_BYTES), dtype=torch.uint8, device="cuda")
    totals = torch.zeros((world, 1), dtype=torch.int32, device="cuda")
    for rank in range(world):
        i0, i1 = shard.coarse_rows(nvc, world, rank)
        a = max(i0 * Fv - 1, 0)                        # the block and its halo rows
        b = min(i1 * Fv + 1, nvc * Fv)
        g.detect_peaks_begin()
        g.detect_peaks_add(P[a:b].contiguous(), i0 * Fv - a, i1 * Fv - a, a, cf)
        g.detect_peaks_end(na, nr0, K, axes=pg, dr_m=R.dr_m, out=lists[rank], n_out=totals[rank])
    merged = g.detect_merge(lists.reshape(-1), totals.reshape(-1), K, K)
    dw, tw = g.decode_detections(*whole, K)
    dm, tm = g.decode_detections(*merged, K)
    assert g.grft_sync_status() == 0
    assert tw == tm and tw > K                         # a real selection among the candidates
    assert dw.tobytes() == dm.tobytes()


def test_merge_rejects_more_records_than_it_sorts(cuda_lib):
    g = cuda_lib
    lists = torch.zeros(3 * 4096 * g._abi.DET_BYTES, dtype=torch.uint8, device="cuda")
    totals = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GrftError):
        g.detect_merge(lists, totals, 4096, 100)       # 3 x 4096 > 8192 records
