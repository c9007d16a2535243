"""Seeded synthetic pulse-compressed echoes (paper Remark 1, eq. received signal_usual).

For each target l with range history R_l(t) = r0_l dr + v_l t + a_l t^2 / 2 (+ b_l t^3 / 6
for an acceleration rate, P = 3):

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


def _dirichlet_positive(x: np.ndarray, N: int) -> np.ndarray:
    """(1/N) sum_{k=0}^{N-1} exp(j 2 pi k x / N): the range profile of a unit echo whose
    spectrum covers the positive band k = 0..N-1 (the asinc envelope with its linear phase)."""
    x = np.asarray(x, dtype=np.float64)
    r = x - N * np.rint(x / N)                          # periodic in N
    out = np.ones_like(r, dtype=np.complex128)
    nz = np.abs(r) > 1e-12
    rn = r[nz]
    out[nz] = np.exp(1j * np.pi * (N - 1) * rn / N) * np.sin(np.pi * rn) / (N * np.sin(np.pi * rn / N))
    return out


def make_echo(radar: Radar, targets: Iterable[Target], seed: int, noise: bool = True,
              window: int = 64, envelope: str = "sinc") -> np.ndarray:
    """Return s[M][N] complex64.  envelope='sinc' (default), 'delta' (a unit sample at the
    nearest bin, used by noiseless closed-form tests) or 'asinc' (paper eq. received signal:
    the range IFFT of the discrete positive band f_k = k f_s / N, k = 0..N-1, of the
    frequency-domain echo exp(-j 4 pi (f_k + f_c) R / c) -- a periodic-sinc envelope with the
    extra linear phase, over the whole range axis)."""
    M, N = radar.M, radar.N
    out = np.zeros((M, N), dtype=np.complex128)
    t = np.arange(M, dtype=np.float64) / radar.prf_hz
    lam = radar.wavelength
    for tg in targets:
        R = tg.r0_bins * radar.dr_m + tg.v * t + 0.5 * tg.a * t * t + (tg.b / 6.0) * t * t * t
        x = R / radar.dr_m
        ph = tg.amp * _carrier(R, lam)
        if envelope == "asinc":
            n = np.arange(N, dtype=np.float64)
            out += ph[:, None] * _dirichlet_positive(n[None, :] - x[:, None], N)
            continue
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
