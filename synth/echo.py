"""Seeded synthetic pulse-compressed echoes (paper Remark 1, eq. received signal_usual).

For each target l with range history R_l(t) = r0_l dr + v_l t + a_l t^2 / 2:

    s[m][n] = sum_l A_l sinc(n - R_l(t_m)/dr) exp(-j 4 pi R_l(t_m) / lambda) + w[m][n]

with f_s = B (so the sinc argument is in bins), noise w ~ CN(0, 1) (re and im each
N(0, 1/2)) drawn from numpy's PCG64 stream for the given seed, and the sinc truncated
to |n - x| <= window bins.  The carrier phase is formed from the FP64 cycle count
2R/lambda reduced modulo one cycle before the exponential.

Output: complex64 array of shape [M][N] (range fastest), the layout the library takes.
"""
from __future__ import annotations

import math
from typing import Iterable

import numpy as np

from .configs import Radar, Target


def _carrier(R: np.ndarray, lam: float) -> np.ndarray:
    u = 2.0 * R / lam
    frac = u - np.rint(u)
    return np.exp(-2j * np.pi * frac)


def make_echo(radar: Radar, targets: Iterable[Target], seed: int, noise: bool = True,
              window: int = 64, envelope: str = "sinc") -> np.ndarray:
    """Return s[M][N] complex64.  envelope='sinc' (default) or 'delta' (a unit sample
    at the nearest bin, used by noiseless closed-form tests)."""
    M, N = radar.M, radar.N
    out = np.zeros((M, N), dtype=np.complex128)
    t = np.arange(M, dtype=np.float64) / radar.prf_hz
    lam = radar.wavelength
    for tg in targets:
        R = tg.r0_bins * radar.dr_m + tg.v * t + 0.5 * tg.a * t * t
        x = R / radar.dr_m
        ph = tg.amp * _carrier(R, lam)
        if envelope == "delta":
            n = np.floor(x + 0.5).astype(np.int64)
            ok = (n >= 0) & (n < N)
            out[np.arange(M)[ok], n[ok]] += ph[ok]
            continue
        lo = np.maximum(np.floor(x).astype(np.int64) - window, 0)
        width = 2 * window + 2
        cols = lo[:, None] + np.arange(width)[None, :]
        ok = cols < N
        env = np.sinc(cols - x[:, None])
        rows = np.broadcast_to(np.arange(M)[:, None], cols.shape)
        np.add.at(out, (rows[ok], cols[ok]), (env * ph[:, None])[ok])
    if noise:
        rng = np.random.Generator(np.random.PCG64(seed))
        w = rng.standard_normal((M, N, 2)) * math.sqrt(0.5)
        out += w[..., 0] + 1j * w[..., 1]
    return out.astype(np.complex64)


def make_noise(shape, seed: int) -> np.ndarray:
    """CN(0,1) complex64 noise of the given shape from the PCG64 stream of `seed`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(tuple(shape) + (2,)) * math.sqrt(0.5)
    return (w[..., 0] + 1j * w[..., 1]).astype(np.complex64)
