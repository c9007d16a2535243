"""GPU: seeded trials of the Monte-Carlo detection study (Sec. VI, Exp. 2; `bench.py --pd`)
replayed against the oracle.  For each trial the GPU map (plain GRFT in FP32, DS-GRFT in
split BF16, as the study runs them) goes through the fixed-threshold detector (eq. LRT with
the 3x3x3 local maximum, `detect_peaks` mode 1), and the FP64 oracle map of the same echo
through the oracle's detector; the study's hit decision (a detection within one cell of the
truth on every axis, among the top 64) must agree, and the whole detection sets must be
equal except cells whose decision lies within the measured power error."""
import numpy as np
import pytest
import torch

import bench
import oracle
import synth
from tests.ambiguity import decision_is_ambiguous
from tests.helpers import TOL_FP32, TOL_SPLIT, rel_peak_err

pytestmark = pytest.mark.gpu

K_STUDY = 64        # the study keeps the top 64 detections per trial
K_ALL = 4096        # every detection, for the set comparison


def _decode_idx(idx, na, nr0):
    idx = np.asarray(idx, dtype=np.int64)
    vi, rem = np.divmod(idx, na * nr0)
    ai, n0 = np.divmod(rem, nr0)
    return vi, ai, n0


@pytest.mark.parametrize("snr", [-12.0, -10.0, -8.0])
def test_pd_trials_match_oracle_decisions(cuda_lib, snr):
    g = cuda_lib
    R, ds, _, cf = synth.pd_setup()
    pg = ds.plain_equivalent()
    nv, na = pg.v.count, pg.a.count
    hits = {"grft": [], "dsgrft": []}
    for trial in range(4):
        j, k, n0, s = synth.pd_trial(R, pg, snr, trial)
        echo = torch.from_numpy(s).cuda()
        for name in ("grft", "dsgrft"):
            P = torch.empty((nv, na, R.N), dtype=torch.float32, device="cuda")
            if name == "grft":
                g.grft_plain(R, echo, pg, None, P)
                P64 = np.abs(oracle.grft_plain_full(R, s, pg)) ** 2
                tol = TOL_FP32
            else:
                g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.n_cells, "bf16x3", None, P)
                P64 = np.abs(oracle.dsgrft_full(R, s, ds)) ** 2
                tol = TOL_SPLIT
            Pg = P.cpu().numpy().astype(np.float64)
            assert rel_peak_err(Pg, P64) <= 2 * tol
            dP = Pg - P64
            # the study's decision: top 64 on each side, hit rule of the study
            out, n = g.detect_peaks(P, cf, K_STUDY)
            dets, _ = g.decode_detections(out, n, K_STUDY)
            idx_o, _, _ = oracle.cfar_detect(P64, cf, K_STUDY)
            hit_g = bench.pd_hit(dets["vi"], dets["ai"], dets["n0"], j, k, n0)
            hit_o = bench.pd_hit(*_decode_idx(idx_o, na, R.N), j, k, n0)
            # every detection on both sides
            outa, na_out = g.detect_peaks(P, cf, K_ALL)
            da, tot_g = g.decode_detections(outa, na_out, K_ALL)
            ia, _, tot_o = oracle.cfar_detect(P64, cf, K_ALL)
            assert tot_g < K_ALL and tot_o < K_ALL
            diff = sorted(set(da["idx"].tolist()) ^ set(ia.tolist()))
            bad = [d for d in diff if not decision_is_ambiguous(P64, dP, cf, d)]
            assert not bad, (name, trial, bad)
            if hit_g != hit_o:
                # only a cell within one cell of the truth whose decision is ambiguous can
                # turn a hit into a miss
                vi, ai, nn = _decode_idx(diff, na, R.N)
                near = (np.abs(vi - j) <= 1) & (np.abs(ai - k) <= 1) & (np.abs(nn - n0) <= 1)
                assert near.any(), (name, trial)
            hits[name].append((hit_g, hit_o))
            del P
        assert g.grft_sync_status() == 0
    print(f"SNR {snr} dB, trials 0-3 (GPU, oracle):", hits)
