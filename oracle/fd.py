"""FP64 oracle of the frequency-domain coarse stage (mGIFT: Def. 2, eq. H-RM and eq.
pre-DFM, Alg. 1) — TEST INFRASTRUCTURE ONLY, numpy.

For coarse cell c (centres v_c, a_c) and pulse m, d_c(t_m) = (v_c t) + ((a_c / 2) t^2) in
the FP64 operation order of the bins, delta = d_c(t_m) / dr, and the range spectrum of the
pulse S[m][k] = sum_n s[m][n] exp(-j 2 pi k n / N):

    Z[c][m][n] = (1/N) sum_k S[m][k] exp(+j 2 pi k (n + delta) / N) * exp(j 4 pi d_c / lambda)

with the frequency index k taken in [-N/2, N/2) (reading: the Nyquist bin at -N/2).
H_RM of eq. H-RM at f_k = k f_s / N is exp(j 2 pi k delta / N) because dr = c / (2 f_s):
the band-limited, circular advance of the range profile by delta bins; H_pre-DFM is the
coarse phase.  The fine stage on Z is the same dense sum as in the time-domain form.
Pinned in tests/test_oracle_pins.py (exact circular shift for integer delta, the shift of
a single range frequency in closed form, a direct O(N^2) DFT).
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


def coarse_rm_fd(radar, s, ds, cell_begin: int, cell_count: int) -> np.ndarray:
    """Z[cell][m][j] complex128, j over [r0_begin, r0_begin + r0_count)."""
    s = np.asarray(s).astype(np.complex128)
    M, N = s.shape
    S = np.fft.fft(s, axis=1)                                  # [m][k]
    k = np.fft.fftfreq(N, d=1.0 / N)                           # signed, Nyquist at -N/2
    n = ds.r0_begin + np.arange(ds.r0_count)
    Z = np.zeros((cell_count, M, ds.r0_count), dtype=np.complex128)
    for ci in range(cell_count):
        d = _coarse_displacement(radar, ds, cell_begin + ci)
        delta = d / radar.dr_m
        ramp = np.exp(2j * np.pi * np.outer(delta, k) / N)      # H_RM
        z = np.fft.ifft(S * ramp, axis=1)                      # [m][n]
        Z[ci] = z[:, n] * _range_phase(d, radar.wavelength)[:, None]
    return Z


def dsgrft_rows_fd(radar, s, ds, cell, fine) -> np.ndarray:
    """Y[row][n0] complex128: the fine stage (dense GFT sum with H_DFM of the fine offsets
    and the range phase) on the frequency-domain coarse output, rows (cell, fine)."""
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
            cache[c] = coarse_rm_fd(radar, s, ds, int(c), 1)[0]
        k, q = divmod(int(f), ds.Fa)
        dv = (k - ds.Fv / 2) * (ds.vc.step / ds.Fv)
        da = (q - ds.Fa / 2) * (ds.ac.step / ds.Fa)
        D = _range_phase((dv * t) + ((0.5 * da) * (t * t)), lam)
        Y[r] = e0 * (cache[c] * D[:, None]).sum(axis=0)
    return Y
