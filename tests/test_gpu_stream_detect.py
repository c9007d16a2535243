"""GPU: detection over a map scanned in slabs (Alg. 3's threshold scan over a grid too large
to hold) equals detection over the whole map.

* detect_peaks_begin / add / end over a map cut into uneven slabs with halo rows gives the
  records and total of detect_peaks over the whole map, bit for bit;
* dsgrft_detect (DS-GRFT computed one coarse-v row of cells at a time into two slab buffers,
  each scanned with its neighbours' border rows as halos) gives exactly the records of
  dsgrft over every cell followed by detect_peaks, in every precision, on a small ragged case
  (detections on slab-border rows included) and on the full M=512 workload."""
import numpy as np
import pytest
import torch

import synth
from synth import CFAR, Axis, DSGrid, Radar, Target

pytestmark = pytest.mark.gpu


def _same(g, a, b, K):
    da, ta = g.decode_detections(*a, K)
    db, tb = g.decode_detections(*b, K)
    assert ta == tb
    assert da.tobytes() == db.tobytes()
    return da, ta


@pytest.mark.parametrize("cuts", [[0, 24], [0, 7, 8, 20, 24], [0, 1, 2, 23, 24]])
def test_slabs_with_halos_equal_whole_map(cuda_lib, cuts):
    g = cuda_lib
    rng = np.random.default_rng(len(cuts))
    nv, na, nr0 = 24, 7, 1000
    P = rng.exponential(1.0, size=(nv, na, nr0)).astype(np.float32)
    for _ in range(60):
        P[rng.integers(nv), rng.integers(na), rng.integers(nr0)] = np.float32(rng.uniform(20, 200))
    # peaks on slab borders and an equal pair across one (the index tie-break spans slabs)
    P[7, 3, 500] = np.float32(300.0)
    P[8, 3, 500] = np.float32(300.0)
    P[20, 1, 10] = np.float32(250.0)
    Pd = torch.from_numpy(P).cuda()
    cf = CFAR(2, 16, 1e-3)
    K = 256
    axes = synth.PlainGrid(5, nr0, Axis(-3.0, 0.5, nv), Axis(1.0, 0.25, na))
    whole = g.detect_peaks(Pd, cf, K, axes=axes, dr_m=15.0)
    g.detect_peaks_begin()
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        a, b = max(lo - 1, 0), min(hi + 1, nv)          # the slab and its halo rows
        g.detect_peaks_add(Pd[a:b].contiguous(), lo - a, hi - a, a, cf)
    part = g.detect_peaks_end(na, nr0, K, axes=axes, dr_m=15.0)
    d, total = _same(g, whole, part, K)
    assert total > 20 and g.grft_sync_status() == 0


def _small():
    R = Radar(M=100, N=700, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(17, 300, Axis(-40.0, 18.75, 4), Axis(-2.5, 5.0, 3), 16, 8)
    tg = [Target(137.0, -21.0, 1.2, complex(3.0, -1.0)), Target(268.3, 3.0, -2.0, complex(1.0, 2.0)),
          Target(200.0, -11.0, 0.3, complex(2.0, 0.0))]
    return R, ds, synth.make_echo(R, tg, 3)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16x2"])
def test_dsgrft_detect_equals_whole_map_small(cuda_lib, precision):
    g = cuda_lib
    R, ds, s = _small()
    echo = torch.from_numpy(s).cuda()
    pg = ds.plain_equivalent()
    cf = CFAR(2, 16, 1e-2)              # many detections, on every slab row
    K = 2048
    P = g.dsgrft(R, echo, ds, precision=precision)
    whole = g.detect_peaks(P, cf, K, axes=pg, dr_m=R.dr_m)
    streamed = g.dsgrft_detect(R, echo, ds, precision, cf, K)
    d, total = _same(g, whole, streamed, K)
    assert g.grft_sync_status() == 0
    border = np.isin(d["vi"] % ds.Fv, [0, ds.Fv - 1])
    assert total < K and border.sum() >= 5          # the halo rows decided some detections


def test_dsgrft_detect_single_coarse_row(cuda_lib):
    g = cuda_lib
    R, ds, s = _small()
    ds = DSGrid(ds.r0_begin, ds.r0_count, Axis(-10.0, 18.75, 1), ds.ac, ds.Fv, ds.Fa)
    echo = torch.from_numpy(s).cuda()
    cf = CFAR(2, 16, 1e-2)
    P = g.dsgrft(R, echo, ds, precision="bf16x3")
    whole = g.detect_peaks(P, cf, 512, axes=ds.plain_equivalent(), dr_m=R.dr_m)
    _same(g, whole, g.dsgrft_detect(R, echo, ds, "bf16x3", cf, 512), 512)


def test_dsgrft_detect_full_ds_m512(cuda_lib):
    """The benchmark workload (2^30 hypotheses): streamed detection over 32 slabs equals the
    whole 4 GiB map's detection, top 1000 records and total."""
    g = cuda_lib
    sc = synth.ds_m512()
    R, ds = sc.radar, sc.ds
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).cuda()
    cf = CFAR(2, 16, 1e-6)
    K = 1000
    P = g.dsgrft(R, echo, ds, precision="fp16x2")
    whole = g.detect_peaks(P, cf, K, axes=ds.plain_equivalent(), dr_m=R.dr_m)
    torch.cuda.synchronize()
    del P
    torch.cuda.empty_cache()
    d, total = _same(g, whole, g.dsgrft_detect(R, echo, ds, "fp16x2", cf, K), K)
    print("ds_m512 streamed detection: total", total)
    assert total > 100 and g.grft_sync_status() == 0
