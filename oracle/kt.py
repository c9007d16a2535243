"""FP64 oracle of the keystone-transform branch, DS-KT-MFP (Sec. III-B eqs. velocity_Amb,
Echo-after-KT, H-MFP, H-MFP-RM, KT-GRFT-GRFT; Sec. IV eq. Partition-Parameter-c1,
Cor. 1, Prop. 3, Alg. 4) — TEST INFRASTRUCTURE ONLY, numpy.

Range spectrum of pulse m: y[m][k] = sum_n s[m][n] exp(-j 2 pi k n / N), with the signed
range frequency f_k = k_s f_s / N, k_s in [-N/2, N/2) (Nyquist at -N/2), f_s = c / (2 dr),
and fbar_k = f_c / (f_c + f_k).

Keystone transform (eq. Echo-after-KT): each range-frequency column is resampled in slow
time at t = fbar_k t'.  Reading: the slow-time sequence is interpolated as a band-limited
periodic sequence of M samples (its M-point DFT, Doppler index l in [-M/2, M/2)):

    Y_k[l]       = sum_m y[m][k] exp(-j 2 pi l m / M)
    y_KT[m'][k]  = (1/M) sum_l Y_k[l] exp(+j 2 pi l fbar_k m' / M)

which is exact for a Doppler tone on the M-point grid.

Coarse stage of DS-KT-MFP (Cor. 1, mGIFT of eq. Definition-modified-GIFT with H_KT,RM and
the KT-MFP H_pre-DFM), coarse cell = (q, c_2,c) with vq = q V_a the cell's velocity centre
(V_a = lambda PRF / 2, eq. velocity_Amb) and c_2,c = a_c / 2:

    Z[c][m][n] = (1/N) sum_k y_KT[m][k] exp(+j 2 pi k_s (fbar_k vq t_m - c_2,c t_m^2) / (N dr))
                       exp(+j 2 pi k_s n / N)  *  exp(+j 4 pi c_2,c t_m^2 / lambda)

(H_KT,RM at f_k: (4 pi / c) f_k x = 2 pi k_s x / (N dr)).  Fine stage (Prop. 3, the GFT of
Def. 1 with the baseband velocity c'_1 and the fine acceleration; kappa = 1 as in the
time-domain branch):

    Y(n; c, k, q) = sum_m Z[c][m][n] exp(+j 4 pi (dv_k t_m + da_q t_m^2 / 2) / lambda)

with dv_k = (k - Fv/2) vc.step / Fv (vc.step = V_a, so c'_1 spans [-V_a/2, V_a/2)) and
da_q = (q - Fa/2) ac.step / Fa.  Unlike the GRFT branch, Y carries no range phase of n
(eq. KT-GRFT-GRFT has none).

Pinned in tests/test_oracle_kt_pins.py: the zero-frequency column is left unchanged (fbar
= 1); an on-grid Doppler tone comes out as the tone at the rescaled time; a target built
from the post-KT signal model (eq. Echo-after-KT) gives |Y| = M at its hypothesis; with
f_c -> infinity and one zero-acceleration cell the whole chain is the range profile's
slow-time DFT (moving-target detection); a physical echo of a target several blind
speeds fast, migrating many bins, is focused to its bins by the keystone branch and not
without the transform.
"""
from __future__ import annotations

import numpy as np


def _signed(n: int) -> np.ndarray:
    return np.fft.fftfreq(n, d=1.0 / n)                       # [0..n/2-1, -n/2..-1]


def _range_phase(x, lam):
    u = 2.0 * x / lam
    return np.exp(2j * np.pi * (u - np.rint(u)))              # exp(j 4 pi x / lambda)


def fbar(radar) -> np.ndarray:
    """fbar_k = f_c / (f_c + f_k) in FFT order (k = 0..N-1, signed frequency)."""
    fs = radar.c_mps / (2.0 * radar.dr_m)
    fk = _signed(radar.N) * fs / radar.N
    return radar.fc_hz / (radar.fc_hz + fk)


def blind_speed(radar) -> float:
    """V_a = lambda PRF / 2 (eq. velocity_Amb)."""
    return radar.wavelength * radar.prf_hz / 2.0


def keystone_columns(radar, s, cols) -> np.ndarray:
    """y_KT[m'][j] complex128 for the range-frequency columns cols[j] (FFT order)."""
    s = np.asarray(s).astype(np.complex128)
    M = s.shape[0]
    cols = np.asarray(cols, dtype=np.int64).ravel()
    n = np.arange(s.shape[1])
    y = s @ np.exp(-2j * np.pi * np.outer(n, cols) / s.shape[1])   # [m][j] range spectrum
    Yd = np.fft.fft(y, axis=0)                                      # [l][j], l in FFT order
    l = _signed(M)
    mp = np.arange(M, dtype=np.float64)
    fb = fbar(radar)[cols]
    out = np.empty((M, cols.size), dtype=np.complex128)
    for j in range(cols.size):
        E = np.exp(2j * np.pi * np.outer(mp, l) * fb[j] / M) / M
        out[:, j] = E @ Yd[:, j]
    return out


def keystone(radar, s) -> np.ndarray:
    """y_KT[m'][k] complex128 for all columns (FFT order along k)."""
    return keystone_columns(radar, s, np.arange(np.asarray(s).shape[1]))


def _cell_params(ds, cell):
    i, l = divmod(int(cell), ds.ac.count)
    return ds.vc.start + i * ds.vc.step, ds.ac.start + l * ds.ac.step


def kt_coarse_rm(radar, ykt, ds, cell_begin: int, cell_count: int) -> np.ndarray:
    """Z[cell][m][j] complex128 (j over the range window) from the post-KT spectra
    ykt[m][k] (FFT order)."""
    ykt = np.asarray(ykt).astype(np.complex128)
    M, N = ykt.shape
    ks = _signed(N)
    fb = fbar(radar)
    t = np.arange(M, dtype=np.float64) / radar.prf_hz
    n = ds.r0_begin + np.arange(ds.r0_count)
    Z = np.empty((cell_count, M, ds.r0_count), dtype=np.complex128)
    for ci in range(cell_count):
        vq, ac = _cell_params(ds, cell_begin + ci)
        c2 = 0.5 * ac
        x = np.outer(vq * t, ks * fb) - np.outer(c2 * (t * t), ks)   # [m][k], metres x k_s
        H = np.exp(2j * np.pi * x / (N * radar.dr_m))                 # H_KT,RM
        z = np.fft.ifft(ykt * H, axis=1)                              # (1/N) sum_k ... e^{+j2pi k n/N}
        Z[ci] = z[:, n] * _range_phase(c2 * (t * t), radar.wavelength)[:, None]   # H_pre-DFM
    return Z


def kt_fine_rows(radar, Zc, ds, fine) -> np.ndarray:
    """Y[row][j] complex128: the fine stage on one cell's coarse output Zc[m][j] for the
    fine indices fine[row] = k * Fa + q."""
    fine = np.asarray(fine).ravel()
    t = np.arange(radar.M, dtype=np.float64) / radar.prf_hz
    Y = np.empty((fine.size, Zc.shape[1]), dtype=np.complex128)
    for r, f in enumerate(fine):
        k, q = divmod(int(f), ds.Fa)
        dv = (k - ds.Fv / 2) * (ds.vc.step / ds.Fv)
        da = (q - ds.Fa / 2) * (ds.ac.step / ds.Fa)
        D = _range_phase((dv * t) + ((0.5 * da) * (t * t)), radar.wavelength)
        Y[r] = (Zc * D[:, None]).sum(axis=0)
    return Y


def dskt_rows(radar, s, ds, cell, fine) -> np.ndarray:
    """Y[row][j] complex128 for hypotheses (cell[row], fine[row]) from the echo s[m][n]."""
    cell = np.asarray(cell).ravel()
    fine = np.asarray(fine).ravel()
    ykt = keystone(radar, s)
    Y = np.empty((cell.size, ds.r0_count), dtype=np.complex128)
    cache = {}
    for r, (c, f) in enumerate(zip(cell, fine)):
        if c not in cache:
            cache[c] = kt_coarse_rm(radar, ykt, ds, int(c), 1)[0]
        Y[r] = kt_fine_rows(radar, cache[c], ds, [f])[0]
    return Y


def dskt_map(radar, s, ds, ykt=None) -> np.ndarray:
    """The whole map Y[v][a][r0] complex128 in the canonical dual-scale layout:
    v index = i Fv + k (cell velocity row i, baseband bin k), a index = l Fa + q."""
    if ykt is None:
        ykt = keystone(radar, s)
    nv, na = ds.vc.count, ds.ac.count
    out = np.empty((nv * ds.Fv, na * ds.Fa, ds.r0_count), dtype=np.complex128)
    t = np.arange(radar.M, dtype=np.float64) / radar.prf_hz
    k = np.arange(ds.Fv)
    q = np.arange(ds.Fa)
    dv = (k - ds.Fv / 2) * (ds.vc.step / ds.Fv)
    da = (q - ds.Fa / 2) * (ds.ac.step / ds.Fa)
    D = _range_phase((dv[:, None, None] * t) + ((0.5 * da)[None, :, None] * (t * t)), radar.wavelength)
    for c in range(nv * na):
        i, l = divmod(c, na)
        Zc = kt_coarse_rm(radar, ykt, ds, c, 1)[0]                   # [m][j]
        Yc = np.einsum("kqm,mj->kqj", D, Zc)
        out[i * ds.Fv:(i + 1) * ds.Fv, l * ds.Fa:(l + 1) * ds.Fa] = Yc
    return out
