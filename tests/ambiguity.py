"""Which detection decisions two correct evaluations of the same power map may disagree on.

The detector of the library and of the oracle (a CA-CFAR threshold along r0, or a fixed
threshold, plus a 3x3x3 local maximum) takes hard decisions on P.  A GPU map differs from
the FP64 map by its rounding error dP, so a cell whose decision margin in the FP64 map is no
larger than the bound dP puts on that margin may be decided either way; every other cell
must be decided identically.  Test infrastructure only."""
import numpy as np


def decision_is_ambiguous(P64, dP, cfar, idx) -> bool:
    """True if the threshold or local-maximum decision of cell idx (linear index
    (vi * na + ai) * nr0 + n0 of P64) can flip under the perturbation dP (GPU map minus the
    FP64 map)."""
    nv, na, nr0 = P64.shape
    vi, rem = divmod(int(idx), na * nr0)
    ai, n = divmod(rem, nr0)
    row, drow = P64[vi, ai], np.abs(dP[vi, ai])
    if cfar.mode == 1:
        if abs(row[n] - cfar.fixed_thresh) <= drow[n] + 1e-6 * abs(cfar.fixed_thresh):
            return True
    else:
        G, T = cfar.guard, cfar.train
        tr = [j for j in list(range(n - G - T, n - G)) + list(range(n + G + 1, n + G + T + 1)) if 0 <= j < nr0]
        if tr:
            k = cfar.pfa ** (-1.0 / len(tr)) - 1.0          # threshold = k * sum of the training cells
            if abs(row[n] - k * row[tr].sum()) <= drow[n] + k * drow[tr].sum():
                return True
    sl = (slice(max(vi - 1, 0), vi + 2), slice(max(ai - 1, 0), ai + 2), slice(max(n - 1, 0), n + 2))
    nb, dnb = P64[sl].ravel(), np.abs(dP[sl]).ravel()
    own = np.ravel_multi_index((vi - sl[0].start, ai - sl[1].start, n - sl[2].start), P64[sl].shape)
    mask = np.arange(nb.size) != own
    return bool(np.any(np.abs(nb[mask] - row[n]) <= dnb[mask] + drow[n]))
