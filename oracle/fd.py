"""FP64 oracle of the frequency-domain coarse stage (mGIFT: Def. 2, eq. H-RM and eq.
pre-DFM, Alg. 1) — TEST INFRASTRUCTURE ONLY, numpy.

For coarse cell c (centres v_c, a_c) and pulse m, d_c(t_m) = (v_c t) + ((a_c / 2) t^2) in
the FP64 operation order of the bins, delta = d_c(t_m) / dr, and the range spectrum of the
pulse S[m][k] = sum_n s[m][n] exp(-j 2 pi k n / N):

    Z[c][m][n] = (1/N) sum_k S[m][k] exp(+j 2 pi k (n + delta) / N) * exp(j 4 pi d_c / lambda)

with the frequency index k taken in [-N/2, N/2) (reading: the Nyquist bin at -N/2), or,
as the paper's echo model has it (eq. Rx-OFDM-Fre1: K_valid = N bins f_k = k f_s / N), in
[0, N) ('positive' band).  After a positive-band coarse stage the residual range term of
the fine offsets leaves a phase proportional to the fine offsets scaled by a factor
(Prop. 1's kappa; see fine_scale for its sign): the fine stage then uses the scaled
offsets.
H_RM of eq. H-RM at f_k = k f_s / N is exp(j 2 pi k delta / N) because dr = c / (2 f_s):
the band-limited, circular advance of the range profile by delta bins; H_pre-DFM is the
coarse phase.  The fine stage on Z is the same dense sum as in the time-domain form.
Pinned in tests/test_oracle_pins.py (exact circular shift for integer delta, the shift of
a single range frequency in closed form in both bands, a direct O(N^2) DFT, the
positive-band echo's spectrum, and the fine scale recovering the coherence a
fine-cell-edge target loses without it).
"""
from __future__ import annotations

import numpy as np


def _coarse_displacement(radar, ds, cell):
    i, l = divmod(int(cell), ds.ac.count)
    vc = ds.vc.start + i * ds.vc.step
    ac = ds.ac.start + l * ds.ac.step
    t = np.arange(radar.M, dtype=np.float64) / radar.prf_hz
    return (vc * t) + ((0.5 * ac) * (t * t))


def _range_phase(x, lam):
    u = 2.0 * x / lam
    return np.exp(2j * np.pi * (u - np.rint(u)))


def _freq_index(N: int, band: str) -> np.ndarray:
    if band == "baseband":
        return np.fft.fftfreq(N, d=1.0 / N)                    # signed, Nyquist at -N/2
    if band == "positive":
        return np.arange(N, dtype=np.float64)                  # f_k = k f_s / N, k = 0..N-1
    raise ValueError(band)


def coarse_rm_fd(radar, s, ds, cell_begin: int, cell_count: int, band: str = "baseband") -> np.ndarray:
    """Z[cell][m][j] complex128, j over [r0_begin, r0_begin + r0_count).  band: the range
    frequencies the spectrum index k stands for -- 'baseband' (k in [-N/2, N/2)) or
    'positive' (the paper's discrete band k = 0..N-1 of eq. Rx-OFDM-Fre1)."""
    s = np.asarray(s).astype(np.complex128)
    M, N = s.shape
    S = np.fft.fft(s, axis=1)                                  # [m][k]
    k = _freq_index(N, band)
    n = ds.r0_begin + np.arange(ds.r0_count)
    Z = np.zeros((cell_count, M, ds.r0_count), dtype=np.complex128)
    for ci in range(cell_count):
        d = _coarse_displacement(radar, ds, cell_begin + ci)
        delta = d / radar.dr_m
        ramp = np.exp(2j * np.pi * np.outer(delta, k) / N)      # H_RM
        z = np.fft.ifft(S * ramp, axis=1)                      # [m][n]
        Z[ci] = z[:, n] * _range_phase(d, radar.wavelength)[:, None]
    return Z


def fine_scale(radar, band: str) -> float:
    """Factor of the fine offsets in H_DFM after a coarse stage over `band`.  Baseband: 1.
    Positive band: the residual range term c_f t^p of a DS-GRFT cell, transformed over
    f_k in [0, B_r), leaves the phase -(4 pi / lambda) (1 + B_r / (2 f_c)) c_f t^p at the
    peak bin (the asinc term's linear phase, eq. received signal, adds to the carrier's);
    Prop. 1 prints kappa = 1 - B_r / (2 f_c), the factor of the keystone branch (Cor. 1),
    whose residual range term enters with the opposite sign.  B_r = f_s = c / (2 dr)."""
    if band == "baseband":
        return 1.0
    if band == "positive":
        return 1.0 + (radar.c_mps / (2.0 * radar.dr_m)) / (2.0 * radar.fc_hz)
    raise ValueError(band)


def dsgrft_rows_fd(radar, s, ds, cell, fine, band: str = "baseband", kap: float = 1.0) -> np.ndarray:
    """Y[row][n0] complex128: the fine stage (dense GFT sum with H_DFM of the fine offsets
    and the range phase) on the frequency-domain coarse output, rows (cell, fine).  kap
    scales the fine offsets in H_DFM (fine_scale(radar, band) restores the coherence of a
    positive-band coarse stage, Prop. 1)."""
    cell = np.asarray(cell).ravel()
    fine = np.asarray(fine).ravel()
    lam = radar.wavelength
    t = np.arange(radar.M, dtype=np.float64) / radar.prf_hz
    n0 = ds.r0_begin + np.arange(ds.r0_count)
    e0 = _range_phase(n0 * radar.dr_m, lam)
    Y = np.zeros((cell.size, ds.r0_count), dtype=np.complex128)
    cache = {}
    for r, (c, f) in enumerate(zip(cell, fine)):
        if c not in cache:
            cache[c] = coarse_rm_fd(radar, s, ds, int(c), 1, band)[0]
        k, q = divmod(int(f), ds.Fa)
        dv = kap * ((k - ds.Fv / 2) * (ds.vc.step / ds.Fv))
        da = kap * ((q - ds.Fa / 2) * (ds.ac.step / ds.Fa))
        D = _range_phase((dv * t) + ((0.5 * da) * (t * t)), lam)
        Y[r] = e0 * (cache[c] * D[:, None]).sum(axis=0)
    return Y
