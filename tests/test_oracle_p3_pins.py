"""Pins of the P = 3 (acceleration-rate) DS-GRFT oracle against values the mathematics
fixes and against independent code."""
import cmath
import math

import numpy as np

import oracle
from oracle.p3 import dsgrft3_rows
from synth import Axis, DSGrid, DSGrid3, Radar, Target
import synth


def test_trivial_b_axis_equals_the_p2_oracle():
    """With one b cell centred at 0 and one fine b offset of 0 the P = 3 sums are the P = 2
    sums of the C oracle."""
    R = Radar(M=48, N=200, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    s = synth.make_echo(R, [Target(80.3, -40.0, 3.0, complex(2.0, 1.0))], 5)
    ds = DSGrid(10, 150, Axis(-50.0, 20.0, 3), Axis(-4.0, 4.0, 2), 4, 2)
    ds3 = DSGrid3(10, 150, ds.vc, ds.ac, Axis(0.0, 0.0, 1), 4, 2, 1)
    rng = np.random.default_rng(2)
    cell = rng.integers(0, ds.n_cells, 12)
    fine = rng.integers(0, ds.n_fine, 12)
    Y3 = dsgrft3_rows(R, s, ds3, cell, fine)         # (i na + l) nb + 0 == i na + l; f == (k Fa + q)
    Y2 = oracle.dsgrft_rows(R, s, ds, cell, fine)
    np.testing.assert_allclose(Y3, Y2, rtol=0, atol=1e-10 * np.abs(Y2).max())


def test_delta_target_at_a_hypothesis_sums_to_M_A():
    R = Radar(M=64, N=256, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    ds3 = DSGrid3(0, 256, Axis(-20.0, 40.0, 2), Axis(-2.0, 4.0, 2), Axis(-24.0, 16.0, 4), 4, 2, 4)
    cell, fine = 1 * 8 + 1 * 4 + 3, 1 * 8 + 0 * 4 + 3            # c = (1, 1, 3), f = (1, 0, 3)
    v, a, b = oracle.p3.cell_centre(ds3, cell)
    dv, da, db = oracle.p3.fine_offsets(ds3, fine)
    A = complex(0.6, -0.8)
    s = synth.make_echo(R, [Target(100.0, v + dv, a + da, A, b + db)], 0, noise=False, envelope="delta")
    Y = dsgrft3_rows(R, s, ds3, [cell], [fine])[0]
    assert abs(Y[100] - R.M * A) < 1e-6 * R.M                          # complex64 echo


def test_brute_force_on_tiny_shapes():
    """Independent pure-Python loops (scalar math, explicit rounding)."""
    R = Radar(M=8, N=32, fc_hz=1.5e9, prf_hz=1000.0, dr_m=15.0)
    rng = np.random.default_rng(7)
    s = rng.standard_normal((R.M, R.N)) + 1j * rng.standard_normal((R.M, R.N))
    ds3 = DSGrid3(3, 20, Axis(-900.0, 1500.0, 2), Axis(-300.0, 500.0, 2), Axis(-4e4, 6e4, 2), 2, 2, 2)
    lam = R.c_mps / R.fc_hz
    rows = [(c, f) for c in range(8) for f in range(8)]
    Y = dsgrft3_rows(R, s, ds3, [r[0] for r in rows], [r[1] for r in rows])
    for r, (c, f) in enumerate(rows):
        i, l, w = c // 4, (c // 2) % 2, c % 2
        k, q, u = f // 4, (f // 2) % 2, f % 2
        vc = ds3.vc.start + i * ds3.vc.step
        ac = ds3.ac.start + l * ds3.ac.step
        bc = ds3.bc.start + w * ds3.bc.step
        dv = (k - 1) * ds3.vc.step / 2
        da = (q - 1) * ds3.ac.step / 2
        db = (u - 1) * ds3.bc.step / 2
        for j in range(ds3.r0_count):
            n0 = ds3.r0_begin + j
            acc = 0j
            for m in range(R.M):
                tm = m / R.prf_hz
                dc = vc * tm + 0.5 * ac * tm * tm + bc / 6.0 * tm * tm * tm
                n = n0 + math.floor(dc / R.dr_m + 0.5)
                if 0 <= n < R.N:
                    df = dv * tm + 0.5 * da * tm * tm + db / 6.0 * tm * tm * tm
                    acc += s[m, n] * cmath.exp(4j * math.pi * (n0 * R.dr_m + dc + df) / lam)
            assert abs(acc - Y[r, j]) < 1e-8 * max(1.0, abs(acc)), (c, f, j)


def test_acceleration_rate_is_focused_by_its_own_b_cell():
    """A noiseless sinc target with b = +24 m/s^3 (a b cell centre) and its (v, a) on a cell
    centre: its hypothesis sums to nearly M |A|; the same (v, a) in the mirrored b cell
    (b = -24: about 34 rad of phase error over the 0.512 s CPI) does not."""
    sc = synth.ds3_m512()
    R, ds3 = sc.radar, sc.ds3
    i, l = 3, 5
    w_pos, w_neg = 3, 0                                             # b centres +24 and -24
    fine = (ds3.Fv // 2) * ds3.Fa * ds3.Fb + (ds3.Fa // 2) * ds3.Fb + ds3.Fb // 2   # zero offsets
    cpos = (i * ds3.ac.count + l) * ds3.bc.count + w_pos
    cneg = (i * ds3.ac.count + l) * ds3.bc.count + w_neg
    v, a, b = oracle.p3.cell_centre(ds3, cpos)
    assert b == 24.0
    s = synth.make_echo(R, [Target(2000.0, v, a, complex(1.0, 0.0), b)], 0, noise=False)
    Y = dsgrft3_rows(R, s, ds3, [cpos, cneg], [fine, fine])
    assert abs(Y[0, 2000]) > 0.95 * R.M
    assert np.abs(Y[1]).max() < 0.3 * R.M
