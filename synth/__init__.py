"""Seeded synthetic inputs (radar parameters, search grids, echoes) shared by the tests,
the oracle runs and the benchmark.  Holds no part of the transform's arithmetic."""
from .configs import (Axis, CFAR, DSGrid, DSGrid3, ds3_m512, PlainGrid, Radar, Scenario, Target, plain_m64, ds_m512, ds_precision_m2048,
                      ds_batch, ds_adjoint_m1024, walk_margin_bins, kt_grid, dskt_m64, dskt_m512)
from .echo import make_echo, make_noise
from .pd import PD_PFA, pd_setup, pd_trial

__all__ = ["Axis", "CFAR", "DSGrid", "DSGrid3", "ds3_m512", "PlainGrid", "Radar", "Scenario", "Target", "plain_m64", "ds_m512",
           "ds_precision_m2048", "ds_batch", "ds_adjoint_m1024", "walk_margin_bins", "kt_grid", "dskt_m64", "dskt_m512", "make_echo", "make_noise",
           "PD_PFA", "pd_setup", "pd_trial"]
