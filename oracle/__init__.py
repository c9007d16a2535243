"""FP64 CPU oracle of the GRFT / DS-GRFT hot path — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library:
  * ``grft_oracle.c``  literal FP64 loops (plain GRFT, coarse RM gather, DS-GRFT,
    CA-CFAR + top-K, trajectory adjoint, refinement), built with gcc
    ``-O2 -fopenmp -ffp-contract=off`` so that every FP64 operation rounds once;
  * ``brute.py``       an independent pure-numpy restatement for tiny shapes;
  * ``fd.py``          the frequency-domain coarse stage (mGIFT with H_RM as a range-
    spectrum phase ramp) and the fine stage on its output, numpy FFT in FP64;
  * ``p3.py``          DS-GRFT with the acceleration rate (P = 3), numpy FP64;
  * ``kt.py``          the keystone transform and the DS-KT-MFP coarse (H_KT,RM) and fine
    stages, numpy FFT and direct sums in FP64.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
tests/test_oracle_pins.py and tests/test_oracle_kt_pins.py (closed forms, library routines, brute force, invariants);
none is "parity unpinned".
"""
from .fd import coarse_rm_fd, dsgrft_rows_fd, fine_scale
from .p3 import dsgrft3_rows
from .kt import blind_speed, dskt_map, dskt_rows, fbar, keystone, keystone_columns, kt_coarse_rm, kt_fine_rows
from .wrap import (bins_phases, coarse_rm, cfar_detect, dsgrft_rows, dsgrft_full, grft_plain_rows,
                   grft_plain_full, load, num_threads, refine, trajectory_grad)

__all__ = ["dsgrft3_rows", "blind_speed", "dskt_map", "dskt_rows", "fbar", "keystone", "keystone_columns", "kt_coarse_rm",
           "kt_fine_rows", "fine_scale", "bins_phases", "coarse_rm", "coarse_rm_fd", "cfar_detect", "dsgrft_rows", "dsgrft_rows_fd",
           "dsgrft_full",
           "grft_plain_rows", "grft_plain_full", "load", "num_threads", "refine", "trajectory_grad"]
