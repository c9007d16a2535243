"""Shared test utilities (no arithmetic of the method here)."""
import numpy as np


def rel_peak_err(y, ref) -> float:
    """max_i |y_i - ref_i| / max_i |ref_i| (the complex-output error metric)."""
    y = np.asarray(y)
    ref = np.asarray(ref)
    den = np.abs(ref).max()
    return float(np.abs(y - ref).max() / (den if den > 0 else 1.0))


# tolerances: FP32 SIMT paths 1e-5 of peak, split tensor-core paths 2e-3 of peak
TOL_FP32 = 1e-5
TOL_SPLIT = 2e-3
