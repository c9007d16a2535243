"""Seeded synthetic inputs (radar parameters, search grids, echoes) shared by the tests,
the oracle runs and the benchmark.  Holds no part of the transform's arithmetic."""
from .configs import (Axis, CFAR, DSGrid, PlainGrid, Radar, Scenario, Target, cfg1, cfg2, cfg3,
                      cfg4, cfg5, walk_margin_bins)
from .echo import make_echo, make_noise

__all__ = ["Axis", "CFAR", "DSGrid", "PlainGrid", "Radar", "Scenario", "Target", "cfg1", "cfg2",
           "cfg3", "cfg4", "cfg5", "walk_margin_bins", "make_echo", "make_noise"]
