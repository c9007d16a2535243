"""Failure detection without a GPU fault: bounded device-side waits that run out latch
GRFT_ETIMEOUT, the kernel returns, the host reads the status and the context stays usable."""
import numpy as np
import pytest
import torch

import oracle
from tests.helpers import TOL_SPLIT, rel_peak_err
from tests.test_gpu_ds import _small_case

pytestmark = pytest.mark.gpu
ETIMEOUT = -4


def test_wait_on_a_flag_nothing_sets_times_out_and_context_survives(cuda_lib):
    g = cuda_lib
    assert g.grft_sync_status() == 0
    g.grft_selftest_wait(2_000_000)          # about a millisecond of SM cycles
    assert g.grft_sync_status() == ETIMEOUT
    assert g.grft_sync_status() == 0         # the status is cleared once read
    # the context is intact: a normal tensor-core call still gives the right answer
    R, ds, s = _small_case()
    Y = g.dsgrft(R, torch.from_numpy(s).cuda(), ds, precision="bf16x3", want_Y=True, want_P=False)
    assert g.grft_sync_status() == 0
    assert rel_peak_err(Y.cpu().numpy(), oracle.dsgrft_full(R, s, ds)) <= TOL_SPLIT


def test_tensor_core_kernel_unwinds_when_its_waits_run_out(cuda_lib):
    """With a wait limit of a few cycles the warp-specialised kernel's barrier waits run out:
    it latches GRFT_ETIMEOUT, drains its copies and MMAs, frees TMEM and returns; with the
    default limit restored the next call is correct."""
    g = cuda_lib
    R, ds, s = _small_case(seed=8)
    echo = torch.from_numpy(s).cuda()
    g.dsgrft(R, echo, ds, precision="bf16x3")        # sizes the workspace at the normal limit
    assert g.grft_sync_status() == 0
    try:
        g.grft_set_wait_limit(16)
        g.dsgrft(R, echo, ds, precision="bf16x3")
        st = g.grft_sync_status()
    finally:
        g.grft_set_wait_limit(0)
    assert st in (ETIMEOUT, 0)
    Y = g.dsgrft(R, echo, ds, precision="bf16x3", want_Y=True, want_P=False)
    assert g.grft_sync_status() == 0
    assert rel_peak_err(Y.cpu().numpy(), oracle.dsgrft_full(R, s, ds)) <= TOL_SPLIT
