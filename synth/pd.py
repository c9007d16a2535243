"""Seeded inputs of the Monte-Carlo detection-probability study (Sec. VI, Exp. 2): the radar,
the search grids, the detector settings and, per (SNR, trial), one on-grid target plus
CN(0,1) noise.  Every trial is drawn from its own seed, so any trial can be replayed alone
(by the benchmark's study and by the tests that check its decisions against the oracle)."""
from __future__ import annotations

import math

import numpy as np

from .configs import CFAR, Axis, DSGrid, Radar, Target, kt_grid, walk_margin_bins
from .echo import make_echo

PD_PFA = 1e-6          # per-cell false-alarm rate of the fixed threshold


def pd_setup():
    """(radar, DS grid, keystone grid, detector).  M=256 x N=512, f_c 1.5 GHz, PRF 1 kHz;
    coarse 8 v x 2 a cells, fine 64 x 8 (512 v x 16 a x 512 r0 hypotheses, residual range
    migration 3.5 m <= dr / 2); the keystone grid (q in [-1, 1], 256 baseband bins of
    V_a / 256 = the DS fine velocity step) holds every DS hypothesis.  Detector: the fixed
    threshold -M ln(PD_PFA) on |Y|^2 (noise alone gives |Y|^2 ~ M Exp(1)) with the 3x3x3
    local maximum."""
    R = Radar(M=256, N=512, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds = DSGrid(0, R.N, Axis(-87.5, 25.0, 8), Axis(-10.0, 20.0, 2), 64, 8)
    ktg = kt_grid(R, -1, 3, ds.ac, ds.Fa, 256)
    cfar = CFAR(2, 16, PD_PFA, fixed_thresh=-R.M * math.log(PD_PFA), mode=1)
    return R, ds, ktg, cfar


def pd_trial(radar: Radar, pg, snr_db: float, trial: int):
    """(j, k, n0, echo) of one trial: a target on the plain grid pg at velocity index j,
    acceleration index k (both off the grid's edges) and range bin n0, with amplitude
    10^(snr/20) and a uniform phase; echo s[M][N] complex64 = the target's sinc-envelope
    echo + CN(0,1) noise (re and im each N(0, 1/2))."""
    rng = np.random.default_rng([7000, int(trial), int(round(1000 * (snr_db + 100)))])
    margin = walk_margin_bins(radar, 100.0, 20.0) + 2
    j = int(rng.integers(1, pg.v.count - 1))
    k = int(rng.integers(1, pg.a.count - 1))
    n0 = int(rng.integers(margin, radar.N - margin))
    amp = complex(10 ** (snr_db / 20) * np.exp(2j * np.pi * rng.uniform()))
    tgt = Target(float(n0), pg.v.start + j * pg.v.step, pg.a.start + k * pg.a.step, amp)
    s = make_echo(radar, [tgt], 0, noise=False).astype(np.complex128)
    w = rng.standard_normal((radar.M, radar.N, 2)) * math.sqrt(0.5)
    s += w[..., 0] + 1j * w[..., 1]
    return j, k, n0, s.astype(np.complex64)
