"""Radar, search-grid and scenario definitions for the seeded synthetic workloads.

This module holds inputs only (sizes, axes, target draws); it contains none of the
transform's arithmetic.  Both the FP64 oracle and the CUDA library consume these
values, and neither imports the other.

Conventions (paper Sec. II-A/II-B, Sec. III-C):
  * c = 3e8 m/s, wavelength lambda = c / f_c.
  * Range bin  dr = c / (2 f_s) with f_s = B (eq. delta-R).
  * Slow time  t_m = m / PRF, m = 0..M-1 (the paper's c_0 is the range at t = 0).
  * Trajectory r(t) = r0 + v t + a t^2 / 2 (eq. slant range with P = 2, c_2 = a/2).
  * Plain grid: r0 = integer bins, v_j = v.start + j v.step, a_k = a.start + k a.step.
  * Dual-scale grid (eqs. Space_c_c, Space_c_f): coarse centres
    v_c(i) = vc.start + i vc.step, fine offsets dv_k = (k - F_v/2) vc.step / F_v,
    k = 0..F_v-1 (half-open, so neighbouring coarse cells do not overlap), and
    likewise for a.  The fine hypothesis set then equals the plain grid with
    v.start = vc.start - vc.step/2 and v.step = vc.step / F_v.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

C_MPS = 3.0e8


@dataclass(frozen=True)
class Radar:
    M: int            # pulses (slow-time samples)
    N: int            # range bins (fast-time samples)
    fc_hz: float      # carrier frequency
    prf_hz: float     # pulse repetition frequency
    dr_m: float       # range bin c / (2 f_s)
    c_mps: float = C_MPS

    @property
    def wavelength(self) -> float:
        return self.c_mps / self.fc_hz

    @property
    def cpi_s(self) -> float:
        return self.M / self.prf_hz


@dataclass(frozen=True)
class Axis:
    start: float
    step: float
    count: int

    def values(self) -> np.ndarray:
        return self.start + np.arange(self.count, dtype=np.float64) * self.step


@dataclass(frozen=True)
class PlainGrid:
    r0_begin: int
    r0_count: int
    v: Axis
    a: Axis

    @property
    def n_hyp(self) -> int:
        return self.r0_count * self.v.count * self.a.count


@dataclass(frozen=True)
class DSGrid:
    r0_begin: int
    r0_count: int
    vc: Axis
    ac: Axis
    Fv: int
    Fa: int

    @property
    def n_cells(self) -> int:
        return self.vc.count * self.ac.count

    @property
    def n_fine(self) -> int:
        return self.Fv * self.Fa

    @property
    def n_hyp(self) -> int:
        return self.r0_count * self.n_cells * self.n_fine

    def plain_equivalent(self) -> PlainGrid:
        """The single-scale grid that searches the same hypotheses."""
        return PlainGrid(
            self.r0_begin, self.r0_count,
            Axis(self.vc.start - 0.5 * self.vc.step, self.vc.step / self.Fv, self.vc.count * self.Fv),
            Axis(self.ac.start - 0.5 * self.ac.step, self.ac.step / self.Fa, self.ac.count * self.Fa),
        )


@dataclass(frozen=True)
class DSGrid3:
    """Dual-scale grid of the P = 3 motion model r = r0 + v t + a t^2/2 + b t^3/6: coarse
    centres vc x ac x bc, fine offsets (k - Fv/2) vc.step/Fv, (q - Fa/2) ac.step/Fa,
    (u - Fb/2) bc.step/Fb.  Cell c = (i na_c + l) nb_c + w, fine f = (k Fa + q) Fb + u."""
    r0_begin: int
    r0_count: int
    vc: Axis
    ac: Axis
    bc: Axis
    Fv: int
    Fa: int
    Fb: int

    @property
    def n_cells(self) -> int:
        return self.vc.count * self.ac.count * self.bc.count

    @property
    def n_fine(self) -> int:
        return self.Fv * self.Fa * self.Fb

    @property
    def n_hyp(self) -> int:
        return self.r0_count * self.n_cells * self.n_fine


@dataclass(frozen=True)
class Target:
    r0_bins: float    # range at t = 0, in bins (may be fractional)
    v: float          # m/s
    a: float          # m/s^2
    amp: complex      # complex amplitude after pulse compression
    b: float = 0.0    # m/s^3, acceleration rate (P = 3; the range gains b t^3 / 6)


@dataclass(frozen=True)
class CFAR:
    guard: int = 2
    train: int = 16
    pfa: float = 1e-6
    fixed_thresh: float = 0.0
    mode: int = 0     # 0: CA-CFAR + 3x3x3 local max; 1: fixed threshold + local max


@dataclass
class Scenario:
    name: str
    radar: Radar
    targets: List[Target]
    seed: int
    plain: PlainGrid | None = None
    ds: DSGrid | None = None
    snr_db: List[float] = field(default_factory=list)
    ds3: "DSGrid3 | None" = None


def _snr_amp(rng: np.random.Generator, snr_db: float) -> complex:
    # per-sample post-compression SNR |A|^2 / sigma^2 with sigma^2 = 1, uniform phase
    mag = 10.0 ** (snr_db / 20.0)
    ph = rng.uniform(0.0, 2.0 * math.pi)
    return complex(mag * math.cos(ph), mag * math.sin(ph))


def walk_margin_bins(radar: Radar, vmax: float, amax: float) -> int:
    T = radar.cpi_s
    return int(math.ceil((vmax * T + 0.5 * amax * T * T) / radar.dr_m)) + 2


def plain_m64(run: int = 0) -> Scenario:
    """Plain GRFT parity case: M=64, N=256, f_c=1 GHz, B=10 MHz (dr=15 m), PRF=500 Hz.

    One sinc-shaped target at r0 = bin 100.3, v = 180 m/s, a = 12 m/s^2, SNR 3 dB.
    Grid 256 r0 x 64 v x 16 a; v_j = 180 + (j-32) lambda/(2T), a_k = 12 + (k-8) lambda/(4T^2).
    """
    radar = Radar(M=64, N=256, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    T = radar.cpi_s
    lam = radar.wavelength
    dv = lam / (2.0 * T)
    da = lam / (2.0 * T * T) * 0.5
    grid = PlainGrid(0, 256, Axis(180.0 - 32 * dv, dv, 64), Axis(12.0 - 8 * da, da, 16))
    seed = 1000 * 1 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    tgt = [Target(100.3, 180.0, 12.0, _snr_amp(rng, 3.0))]
    return Scenario("plain_m64", radar, tgt, seed, plain=grid, snr_db=[3.0])


def _ds_grid_32x8(radar: Radar, Fv: int, Fa: int, r0_count: int | None = None) -> DSGrid:
    # coarse 32 v x 8 a cells tiling v in [-300, 300] m/s, a in [-20, 20] m/s^2 (cell centres)
    vstep = 600.0 / 32
    astep = 40.0 / 8
    return DSGrid(0, radar.N if r0_count is None else r0_count,
                  Axis(-300.0 + 0.5 * vstep, vstep, 32), Axis(-20.0 + 0.5 * astep, astep, 8), Fv, Fa)


def _random_targets(rng: np.random.Generator, radar: Radar, n: int, snr_lo: float, snr_hi: float,
                    vlim: float = 295.0, alim: float = 19.5) -> Tuple[List[Target], List[float]]:
    margin = walk_margin_bins(radar, 300.0, 20.0)
    tg, snrs = [], []
    for _ in range(n):
        r0 = rng.uniform(margin, radar.N - margin)
        v = rng.uniform(-vlim, vlim)
        a = rng.uniform(-alim, alim)
        snr = rng.uniform(snr_lo, snr_hi)
        tg.append(Target(float(r0), float(v), float(a), _snr_amp(rng, snr)))
        snrs.append(float(snr))
    return tg, snrs


def ds_m512(run: int = 0) -> Scenario:
    """DS-GRFT vs plain GRFT: M=512, N=4096, f_c=1.5 GHz, PRF=1 kHz, dr=15 m, 8 targets,
    v in [-300,300] m/s, a in [-20,20] m/s^2, SNR in [-15,0] dB.
    Coarse grid 4096 r0 x 32 v x 8 a; fine 64 dv x 16 da per coarse cell (2^30 hypotheses)."""
    radar = Radar(M=512, N=4096, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    seed = 1000 * 2 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    tg, snrs = _random_targets(rng, radar, 8, -15.0, 0.0)
    ds = _ds_grid_32x8(radar, 64, 16)
    return Scenario("ds_m512", radar, tg, seed, plain=ds.plain_equivalent(), ds=ds, snr_db=snrs)


def ds_precision_m2048(run: int = 0) -> Scenario:
    """Precision case: M=2048, N=8192, 32 targets, SNR in [-20,0] dB, f_c=1.5 GHz, PRF=1 kHz,
    coarse 32 v x 8 a as in ds_m512, fine 256 dv x 64 da (3.4e10 hypotheses)."""
    radar = Radar(M=2048, N=8192, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    seed = 1000 * 3 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    tg, snrs = _random_targets(rng, radar, 32, -20.0, 0.0)
    ds = _ds_grid_32x8(radar, 256, 64)
    return Scenario("ds_precision_m2048", radar, tg, seed, plain=ds.plain_equivalent(), ds=ds, snr_db=snrs)


def ds_batch(run: int = 0, n_cpi: int = 64) -> List[Scenario]:
    """Batching case: n_cpi independent CPIs with M ~ U{256..2048}, N ~ U{1024..8192},
    1-16 targets each at SNR in [-15,5] dB; grids as in ds_m512 (fine 64 x 16)."""
    seed = 1000 * 4 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cpi):
        M = int(rng.integers(256, 2049))
        N = int(rng.integers(1024, 8193))
        radar = Radar(M=M, N=N, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
        nt = int(rng.integers(1, 17))
        tg, snrs = _random_targets(rng, radar, nt, -15.0, 5.0)
        ds = _ds_grid_32x8(radar, 64, 16)
        out.append(Scenario(f"ds_batch[{i}]", radar, tg, seed * 100 + i, plain=ds.plain_equivalent(), ds=ds,
                            snr_db=snrs))
    return out


def ds_adjoint_m1024(run: int = 0) -> Scenario:
    """Differentiation case: M=1024, N=4096, 16 targets whose motion lies off-grid
    (uniform sub-cell offsets); grids as in ds_m512; top-1000 detections, 20 ascent steps."""
    radar = Radar(M=1024, N=4096, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    seed = 1000 * 5 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    ds = _ds_grid_32x8(radar, 64, 16)
    pg = ds.plain_equivalent()
    margin = walk_margin_bins(radar, 300.0, 20.0)
    tg, snrs = [], []
    for _ in range(16):
        j = int(rng.integers(2, pg.v.count - 2))
        k = int(rng.integers(2, pg.a.count - 2))
        n0 = int(rng.integers(margin, radar.N - margin))
        ov, oa, orr = rng.uniform(-0.5, 0.5, size=3)
        snr = float(rng.uniform(-10.0, 0.0))
        tg.append(Target(n0 + float(orr), float(pg.v.start + (j + ov) * pg.v.step),
                         float(pg.a.start + (k + oa) * pg.a.step), _snr_amp(rng, snr)))
        snrs.append(snr)
    return Scenario("ds_adjoint_m1024", radar, tg, seed, plain=pg, ds=ds, snr_db=snrs)


def ds3_m512(run: int = 0) -> Scenario:
    """P = 3 (acceleration rate) on the ds_m512 radar: 4 targets with v in [-70, 70] m/s,
    a in [-9.5, 9.5] m/s^2, b in [-28, 28] m/s^3, SNR in [-10, 0] dB.  Coarse 8 v x 8 a x 4 b
    cells (centres over [-75, 75] m/s, [-10, 10] m/s^2, [-32, 32] m/s^3), fine 64 dv x 8 da
    x 4 db (0.293 m/s, 0.3125 m/s^2, 4 m/s^3): 4096 r0 x 256 cells x 2048 fine = 2.1e9
    hypotheses; residual range migration of a cell 5.2 m <= dr / 2."""
    radar = Radar(M=512, N=4096, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    seed = 1000 * 7 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    margin = walk_margin_bins(radar, 80.0, 10.0) + 2
    tg, snrs = [], []
    for _ in range(4):
        snr = float(rng.uniform(-10.0, 0.0))
        tg.append(Target(float(rng.uniform(margin, radar.N - margin)), float(rng.uniform(-70.0, 70.0)),
                         float(rng.uniform(-9.5, 9.5)), _snr_amp(rng, snr), float(rng.uniform(-28.0, 28.0))))
        snrs.append(snr)
    ds3 = DSGrid3(0, radar.N, Axis(-75.0 + 9.375, 18.75, 8), Axis(-10.0 + 1.25, 2.5, 8), Axis(-24.0, 16.0, 4),
                  64, 8, 4)
    return Scenario("ds3_m512", radar, tg, seed, snr_db=snrs, ds3=ds3)


def kt_grid(radar: Radar, q_min: int, q_count: int, ac: Axis, Fa: int, L: int | None = None,
            r0_begin: int = 0, r0_count: int | None = None) -> DSGrid:
    """Keystone-branch (DS-KT-MFP) grid as a DSGrid: the coarse velocity axis is the folding
    factor, centres q V_a for q = q_min .. q_min + q_count - 1 (V_a = lambda PRF / 2, eq.
    velocity_Amb); the fine velocity is the baseband velocity on L = Fv transform bins of
    V_a / L over [-V_a/2, V_a/2) (eq. Space_baseband_velocity); L defaults to the smallest
    power of two >= M.  Its plain-equivalent velocity axis starts at (q_min - 1/2) V_a."""
    va = radar.wavelength * radar.prf_hz / 2.0
    if L is None:
        L = 1 << max(0, (radar.M - 1).bit_length())
    return DSGrid(r0_begin, radar.N - r0_begin if r0_count is None else r0_count,
                  Axis(q_min * va, va, q_count), ac, L, Fa)


def dskt_m64(run: int = 0) -> Scenario:
    """Keystone-branch parity case on the plain_m64 radar (M=64, N=256, f_c=1 GHz, PRF=500 Hz,
    dr=15 m, V_a=75 m/s): 3 targets with v in [-200, 200] m/s, a in [-15, 15] m/s^2, SNR 10 dB;
    q in [-3, 3], 4 coarse a cells over [-20, 20] m/s^2, Fa=4, L=64."""
    radar = Radar(M=64, N=256, fc_hz=1.0e9, prf_hz=500.0, dr_m=15.0)
    seed = 1000 * 6 + run
    rng = np.random.Generator(np.random.PCG64(seed))
    tg, snrs = _random_targets(rng, radar, 3, 10.0, 10.0, vlim=200.0, alim=15.0)
    ds = kt_grid(radar, -3, 7, Axis(-15.0, 10.0, 4), 4)
    return Scenario("dskt_m64", radar, tg, seed, plain=ds.plain_equivalent(), ds=ds, snr_db=snrs)


def dskt_m512(run: int = 0) -> Scenario:
    """Keystone branch on the ds_m512 echo (same radar, seed and 8 targets): q in [-3, 3]
    (V_a = 100 m/s, so the fine velocity covers [-350, 350) m/s in 3584 bins of 0.195 m/s),
    the coarse a axis of ds_m512 (8 cells of 5 m/s^2), Fa=16, L=512: 4096 r0 x 3584 v x 128 a
    = 1.88e9 hypotheses."""
    base = ds_m512(run)
    ds = kt_grid(base.radar, -3, 7, base.ds.ac, 16, 512)
    return Scenario("dskt_m512", base.radar, base.targets, base.seed, plain=ds.plain_equivalent(), ds=ds,
                    snr_db=base.snr_db)


def scaled(s: Scenario, **radar_overrides) -> Scenario:
    return dataclasses.replace(s, radar=dataclasses.replace(s.radar, **radar_overrides))
