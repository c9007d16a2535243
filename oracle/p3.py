"""FP64 oracle of DS-GRFT with the acceleration rate (P = 3; Sec. II eq. slant range with
c_3 = b / 6, Alg. 3 extended to P > 2 as the paper notes) — TEST INFRASTRUCTURE ONLY, numpy.

Trajectory r(t) = r0 + v t + a t^2 / 2 + b t^3 / 6.  The displacement is evaluated in FP64
in this operation order, each operation rounded once (numpy does not contract):

    d(v, a, b, t) = ((v t) + ((0.5 a) (t t))) + ((b / 6) ((t t) t))

and the bin shift is rho = floor(d / dr + 1/2).  Dual-scale grid (synth.DSGrid3): cell
c = (i na_c + l) nb_c + w with centres (v_c, a_c, b_c), fine f = (k Fa + q) Fb + u with
offsets dv_k = (k - Fv/2) vc.step / Fv (likewise da_q, db_u).  For range bin n0:

    Y(n0; c, f) = e0(n0) sum_m s[m][n0 + rho_c(m)] w_c(m) D_f(m),
    w_c(m) = exp(j 4 pi d(v_c, a_c, b_c, t_m) / lambda),
    D_f(m) = exp(j 4 pi d(dv_k, da_q, db_u, t_m) / lambda),  e0(n0) = exp(j 4 pi n0 dr / lambda)

(samples outside [0, N) contribute zero; phases from FP64 cycle counts reduced mod 1).
Pinned in tests/test_oracle_p3_pins.py: it equals the P = 2 C oracle when the b axis is
trivial, a noiseless delta target at a hypothesis gives |Y| = M |A|, an independent
pure-Python brute force on tiny shapes, and a target with an acceleration rate is focused
by its own b cell and not by the mirrored one.
"""
from __future__ import annotations

import numpy as np


def disp3(v, a, b, t):
    return ((v * t) + ((0.5 * a) * (t * t))) + ((b / 6.0) * ((t * t) * t))


def _phase(x, lam):
    u = 2.0 * x / lam
    return np.exp(2j * np.pi * (u - np.rint(u)))


def cell_centre(ds3, cell):
    i, rest = divmod(int(cell), ds3.ac.count * ds3.bc.count)
    l, w = divmod(rest, ds3.bc.count)
    return (ds3.vc.start + i * ds3.vc.step, ds3.ac.start + l * ds3.ac.step, ds3.bc.start + w * ds3.bc.step)


def fine_offsets(ds3, fine):
    k, rest = divmod(int(fine), ds3.Fa * ds3.Fb)
    q, u = divmod(rest, ds3.Fb)
    return ((k - ds3.Fv / 2) * (ds3.vc.step / ds3.Fv), (q - ds3.Fa / 2) * (ds3.ac.step / ds3.Fa),
            (u - ds3.Fb / 2) * (ds3.bc.step / ds3.Fb))


def coarse3(radar, ds3, cell):
    """(rho[M] int64, w[M] complex128) of a coarse cell."""
    t = np.arange(radar.M, dtype=np.float64) / radar.prf_hz
    v, a, b = cell_centre(ds3, cell)
    d = disp3(v, a, b, t)
    return np.floor(d / radar.dr_m + 0.5).astype(np.int64), _phase(d, radar.wavelength)


def dsgrft3_rows(radar, s, ds3, cell, fine) -> np.ndarray:
    """Y[row][j] complex128 for hypotheses (cell[row], fine[row]), j over the range window."""
    s = np.asarray(s).astype(np.complex128)
    M, N = s.shape
    cell = np.asarray(cell).ravel()
    fine = np.asarray(fine).ravel()
    t = np.arange(M, dtype=np.float64) / radar.prf_hz
    n0 = ds3.r0_begin + np.arange(ds3.r0_count)
    e0 = _phase(n0 * radar.dr_m, radar.wavelength)
    Y = np.empty((cell.size, ds3.r0_count), dtype=np.complex128)
    cache = {}
    for r, (c, f) in enumerate(zip(cell, fine)):
        if c not in cache:
            rho, w = coarse3(radar, ds3, c)
            idx = n0[None, :] + rho[:, None]                              # [m][j]
            ok = (idx >= 0) & (idx < N)
            Z = np.where(ok, s[np.arange(M)[:, None], np.clip(idx, 0, N - 1)], 0.0) * w[:, None]
            cache[c] = Z
        dv, da, db = fine_offsets(ds3, f)
        D = _phase(disp3(dv, da, db, t), radar.wavelength)
        Y[r] = e0 * (cache[c] * D[:, None]).sum(axis=0)
    return Y
