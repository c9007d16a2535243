"""Pins of the keystone-transform oracle (DS-KT-MFP, Sec. III-B, Cor. 1, Prop. 3, Alg. 4)
against values the mathematics and the physics fix, not against its own formulas."""
import numpy as np
import pytest

import oracle
from synth import Axis, DSGrid, Radar

C = 3.0e8


def _radar(M=64, N=256, fc=1.0e9, prf=500.0, dr=15.0):
    return Radar(M=M, N=N, fc_hz=fc, prf_hz=prf, dr_m=dr)


def _fk(radar):
    # signed range frequency of each FFT-order column, f_s = c / (2 dr)
    fs = C / (2.0 * radar.dr_m)
    k = np.arange(radar.N)
    ks = np.where(k < radar.N // 2, k, k - radar.N)
    return ks * fs / radar.N


def _physical_echo(radar, r0_m, v, a):
    """Pulse-compressed echo of one unit point target with range r0 + v t + a t^2 / 2,
    built from its range spectrum exp(-j 4 pi (f_c + f_k) R(t_m) / c) over the band."""
    t = np.arange(radar.M) / radar.prf_hz
    R = r0_m + v * t + 0.5 * a * t * t
    y = np.exp(-4j * np.pi * np.outer(R, radar.fc_hz + _fk(radar)) / C)
    return np.fft.ifft(y, axis=1)


def test_zero_frequency_column_is_unchanged():
    radar = _radar()
    rng = np.random.default_rng(5)
    s = rng.standard_normal((radar.M, radar.N)) + 1j * rng.standard_normal((radar.M, radar.N))
    got = oracle.keystone_columns(radar, s, [0])[:, 0]
    want = s.sum(axis=1)                                      # DC range bin of each pulse
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("k0,l0", [(5, 7), (253, -20), (128, -32), (37, 0)])
def test_on_grid_tone_is_resampled_in_time(k0, l0):
    """A Doppler tone on the M-point grid in one range-frequency column comes out as the
    same tone at time fbar t: exp(j 2 pi l0 fbar m' / M), fbar = f_c / (f_c + f_k)."""
    radar = _radar()
    M, N = radar.M, radar.N
    m = np.arange(M)[:, None]
    n = np.arange(N)[None, :]
    s = np.exp(2j * np.pi * k0 * n / N) / N * np.exp(2j * np.pi * l0 * m / M)
    ykt = oracle.keystone(radar, s)
    fb = radar.fc_hz / (radar.fc_hz + _fk(radar)[k0])
    want = np.exp(2j * np.pi * l0 * fb * np.arange(M) / M)
    assert np.max(np.abs(ykt[:, k0] - want)) < 1e-10
    others = np.delete(ykt, k0, axis=1)
    assert np.max(np.abs(others)) < 1e-10                     # columns do not mix


def _kt_grid(radar, q_min, q_count, ac_start, ac_step, ac_count, Fa, r0_begin=0, r0_count=None):
    va = radar.wavelength * radar.prf_hz / 2.0
    return DSGrid(r0_begin, radar.N if r0_count is None else r0_count,
                  Axis(q_min * va, va, q_count), Axis(ac_start, ac_step, ac_count), radar.M, Fa)


@pytest.mark.parametrize("da_index", [2, 3])
def test_post_kt_model_focuses_to_M(da_index):
    """An input written from the post-keystone signal model (eq. Echo-after-KT, unit
    amplitude) gives |Y| = M exactly at its hypothesis: range bin, folding factor q,
    baseband velocity bin and coarse + fine acceleration.  For a fine acceleration offset
    the model's range term carries the coarse part only (the dual-scale split)."""
    radar = _radar(M=128, N=256, dr=3.0)
    M, N = radar.M, radar.N
    lam = radar.wavelength
    va = lam * radar.prf_hz / 2.0
    ds = _kt_grid(radar, -3, 7, -150.0, 100.0, 4, 4)
    t = np.arange(M) / radar.prf_hz
    fk = _fk(radar)
    fb = radar.fc_hz / (radar.fc_hz + fk)
    n_t, q, kb, cell_a = 101, 2, 100, 3                        # truth: bin, fold, baseband bin, a cell
    c0 = n_t * radar.dr_m
    c1p = (kb - ds.Fv / 2) * va / ds.Fv
    c2c = 0.5 * (ds.ac.start + cell_a * ds.ac.step)
    c2 = c2c + 0.5 * (da_index - ds.Fa / 2) * ds.ac.step / ds.Fa
    ykt = (np.exp(-4j * np.pi * c0 / lam)
           * np.exp(-4j * np.pi / C * fk[None, :] * (c0 + fb[None, :] * q * va * t[:, None]
                                                      - c2c * (t * t)[:, None]))
           * np.exp(-4j * np.pi / lam * (c1p * t + c2 * t * t))[:, None])
    cell = (q + 3) * ds.ac.count + cell_a
    Z = oracle.kt_coarse_rm(radar, ykt, ds, cell, 1)[0]
    Y = oracle.kt_fine_rows(radar, Z, ds, [kb * ds.Fa + da_index, kb * ds.Fa + (da_index ^ 1),
                                            (kb + 1) * ds.Fa + da_index])
    assert abs(abs(Y[0, n_t]) - M) < 1e-9 * M
    assert abs(Y[0, n_t] - M * np.exp(-4j * np.pi * c0 / lam)) < 1e-8 * M
    assert np.max(np.abs(Y[0, np.arange(N) != n_t])) < 1e-8 * M   # other bins: zero (the IFFT)
    assert abs(Y[2, n_t]) < 1e-8 * M                           # next baseband bin: zero (grid DFT)
    assert abs(Y[1, n_t]) < 0.9 * M
    # a neighbouring fold does not focus
    Zo = oracle.kt_coarse_rm(radar, ykt, ds, cell - ds.ac.count, 1)[0]
    Yo = oracle.kt_fine_rows(radar, Zo, ds, [kb * ds.Fa + da_index])
    assert np.max(np.abs(Yo)) < 0.5 * M


def test_infinite_carrier_limit_is_moving_target_detection():
    """With f_c -> infinity every fbar is 1 (the keystone transform is the identity) and
    one cell with q = 0 and zero acceleration leaves the range profile untouched: the map
    is then the slow-time DFT of each range bin (Doppler bin (k - Fv/2) mod M)."""
    radar = _radar(M=32, N=64, fc=1.0e20, prf=500.0)
    ds = _kt_grid(radar, 0, 1, 0.0, 2.0, 1, 2)                 # a_c = 0; fine index 1 -> da = 0
    rng = np.random.default_rng(9)
    s = rng.standard_normal((radar.M, radar.N)) + 1j * rng.standard_normal((radar.M, radar.N))
    Y = oracle.dskt_map(radar, s, ds)                          # [Fv][Fa][N]
    mtd = np.fft.ifft(s, axis=0) * radar.M                     # sum_m s e^{+j 2 pi f m / M}
    idx = (np.arange(ds.Fv) - ds.Fv // 2) % radar.M
    want = mtd[idx]
    assert np.max(np.abs(Y[:, 1, :] - want)) < 1e-9 * np.max(np.abs(want))


def _peak_at(Y, n_t):
    return np.abs(Y[:, n_t]).max()


def test_fast_target_is_focused_by_the_keystone_branch():
    """A point target three blind speeds fast whose echo migrates 44 range bins over the
    CPI: after the keystone transform, the coarse cell of its folding factor and the
    baseband bin of its remaining velocity focus it to nearly M; without the transform
    the baseband part keeps walking (3.8 bins) and the sum loses most of its power."""
    radar = _radar(M=256, N=512, fc=1.0e9, prf=500.0, dr=3.0)
    M = radar.M
    va = radar.wavelength * radar.prf_hz / 2.0
    ds = _kt_grid(radar, 0, 4, 0.0, 40.0, 1, 2)
    kb = ds.Fv // 2 + 77                                       # baseband 0.30 V_a
    v = 3 * va + (kb - ds.Fv / 2) * va / ds.Fv
    n_t = 120
    s = _physical_echo(radar, n_t * radar.dr_m, v, 0.0)
    walk = v * radar.cpi_s / radar.dr_m
    assert walk > 40
    ykt = oracle.keystone(radar, s)
    Z = oracle.kt_coarse_rm(radar, ykt, ds, 3, 1)[0]           # q = 3, a_c = 0
    Y = oracle.kt_fine_rows(radar, Z, ds, [kb * ds.Fa + 1])
    assert abs(Y[0, n_t]) > 0.9 * M
    assert np.argmax(np.abs(Y[0])) == n_t
    # the neighbouring baseband bins and folds are lower
    Yn = oracle.kt_fine_rows(radar, Z, ds, [(kb + 2) * ds.Fa + 1, (kb - 2) * ds.Fa + 1])
    assert np.max(np.abs(Yn[:, n_t])) < 0.5 * abs(Y[0, n_t])
    for cell in (2, 1):
        Zo = oracle.kt_coarse_rm(radar, ykt, ds, cell, 1)[0]
        assert _peak_at(oracle.kt_fine_rows(radar, Zo, ds, [kb * ds.Fa + 1]), n_t) < 0.5 * M
    # without the keystone transform (plain range spectra) the same hypothesis smears
    y = np.fft.fft(s, axis=1)
    Zn = oracle.kt_coarse_rm(radar, y, ds, 3, 1)[0]
    assert np.max(np.abs(oracle.kt_fine_rows(radar, Zn, ds, [kb * ds.Fa + 1]))) < 0.5 * M


def test_accelerating_target_needs_the_post_kt_sign():
    """After the keystone transform the acceleration's range migration enters with the
    opposite sign (eq. Echo-after-KT: c_0 + fbar q V_a t - c_2 t^2).  An accelerating
    target (5 bins of quadratic migration) is focused by the cell of its own acceleration
    and not by the mirrored one."""
    radar = _radar(M=256, N=512, fc=1.0e9, prf=1000.0, dr=1.0)
    M = radar.M
    va = radar.wavelength * radar.prf_hz / 2.0
    ds = _kt_grid(radar, 0, 1, -150.0, 300.0, 2, 2)           # a_c = -150, +150
    kb = ds.Fv // 2 - 33
    c1p = (kb - ds.Fv / 2) * va / ds.Fv                        # centres the Doppler sweep
    a = 150.0
    n_t = 200
    s = _physical_echo(radar, n_t * radar.dr_m, c1p, a)
    assert 0.5 * a * radar.cpi_s ** 2 / radar.dr_m > 4.5
    ykt = oracle.keystone(radar, s)
    Y = oracle.kt_fine_rows(radar, oracle.kt_coarse_rm(radar, ykt, ds, 1, 1)[0], ds, [kb * ds.Fa + 1])
    assert abs(Y[0, n_t]) > 0.7 * M
    assert np.argmax(np.abs(Y[0])) == n_t
    Zm = oracle.kt_coarse_rm(radar, ykt, ds, 0, 1)[0]          # mirrored acceleration
    Ym = oracle.kt_fine_rows(radar, Zm, ds, [kb * ds.Fa + 1])
    assert np.max(np.abs(Ym)) < 0.3 * M
