"""Independent brute-force restatement of the coherent sums in plain numpy, for tiny
shapes only (test infrastructure).  Written separately from grft_oracle.c so that the
two can pin each other: the phase here is taken from the full range r = n0 dr + d at
every (hypothesis, pulse) pair, and the loops over hypotheses are Python loops.

Definitions (paper eq. standard-GRFT-TD, eq. slant range with P = 2, Alg. 3):
  t_m = m / PRF;  d = v t + a t^2 / 2 (FP64, (v*t) + ((0.5*a)*(t*t)));
  bin = n0 + floor(d/dr + 0.5);  phase = exp(+j 4 pi (n0 dr + d) / lambda).
"""
from __future__ import annotations

import numpy as np


def _t(radar):
    return np.arange(radar.M, dtype=np.float64) / radar.prf_hz


def _disp(v, a, t):
    return (v * t) + ((0.5 * a) * (t * t))


def _phase(x, lam):
    u = (2.0 * x) / lam
    f = u - np.rint(u)
    return np.exp(2j * np.pi * f)


def _gather(s, m_idx, n_idx):
    N = s.shape[1]
    ok = (n_idx >= 0) & (n_idx < N)
    out = np.zeros(n_idx.shape, dtype=np.complex128)
    out[ok] = s[m_idx[ok], n_idx[ok]].astype(np.complex128)
    return out


def grft_plain(radar, s, grid) -> np.ndarray:
    t = _t(radar)
    lam = radar.wavelength
    m = np.arange(radar.M)
    out = np.zeros((grid.v.count, grid.a.count, grid.r0_count), dtype=np.complex128)
    for j in range(grid.v.count):
        v = grid.v.start + j * grid.v.step
        for k in range(grid.a.count):
            a = grid.a.start + k * grid.a.step
            d = _disp(v, a, t)
            rho = np.floor(d / radar.dr_m + 0.5).astype(np.int64)
            for jj in range(grid.r0_count):
                n0 = grid.r0_begin + jj
                vals = _gather(s, m, n0 + rho)
                out[j, k, jj] = np.sum(vals * _phase(n0 * radar.dr_m + d, lam))
    return out


def dsgrft(radar, s, ds) -> np.ndarray:
    """Canonical layout Y[i*Fv + k][l*Fa + q][n0]."""
    t = _t(radar)
    lam = radar.wavelength
    m = np.arange(radar.M)
    nv, na = ds.vc.count * ds.Fv, ds.ac.count * ds.Fa
    out = np.zeros((nv, na, ds.r0_count), dtype=np.complex128)
    for i in range(ds.vc.count):
        vc = ds.vc.start + i * ds.vc.step
        for l in range(ds.ac.count):
            ac = ds.ac.start + l * ds.ac.step
            dc = _disp(vc, ac, t)
            rho = np.floor(dc / radar.dr_m + 0.5).astype(np.int64)
            for k in range(ds.Fv):
                dv = (k - ds.Fv / 2.0) * ds.vc.step / ds.Fv
                for q in range(ds.Fa):
                    da = (q - ds.Fa / 2.0) * ds.ac.step / ds.Fa
                    df = _disp(dv, da, t)
                    for jj in range(ds.r0_count):
                        n0 = ds.r0_begin + jj
                        vals = _gather(s, m, n0 + rho)
                        ph = _phase(n0 * radar.dr_m + dc + df, lam)
                        out[i * ds.Fv + k, l * ds.Fa + q, jj] = np.sum(vals * ph)
    return out


def cfar_detect(P, guard, train, pfa, K, mode=0, fixed_thresh=0.0):
    """Python-loop restatement of the CA-CFAR + 3x3x3 local max + top-K rule."""
    nv, na, nr0 = P.shape
    hits = []
    for vi in range(nv):
        for ai in range(na):
            row = P[vi, ai]
            for n in range(nr0):
                tr = [row[j] for j in list(range(n - guard - train, n - guard)) +
                      list(range(n + guard + 1, n + guard + train + 1)) if 0 <= j < nr0]
                if mode == 0:
                    if not tr:
                        continue
                    alpha = len(tr) * (pfa ** (-1.0 / len(tr)) - 1.0)
                    if not row[n] > alpha * (sum(tr) / len(tr)):
                        continue
                elif not row[n] > fixed_thresh:
                    continue
                me = (vi * na + ai) * nr0 + n
                ok = True
                for dv in (-1, 0, 1):
                    for da in (-1, 0, 1):
                        for dn in (-1, 0, 1):
                            if dv == da == dn == 0:
                                continue
                            v2, a2, n2 = vi + dv, ai + da, n + dn
                            if 0 <= v2 < nv and 0 <= a2 < na and 0 <= n2 < nr0:
                                o = (v2 * na + a2) * nr0 + n2
                                if P[v2, a2, n2] > row[n] or (P[v2, a2, n2] == row[n] and o < me):
                                    ok = False
                if ok:
                    hits.append((-row[n], me))
    hits.sort()
    return [h[1] for h in hits[:K]], [-h[0] for h in hits[:K]], len(hits)
