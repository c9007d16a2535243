"""One CPI's DS-GRFT search split over the GPUs of a job (one process per GPU).

The coarse cells of Alg. 3 are independent, so the grid is cut between the ranks along the
coarse velocity axis: rank r computes the power map of coarse-v rows [i0, i1) (whole rows
of cells, every fine hypothesis, every r0 bin) on its own GPU from its own copy of the echo.
The threshold scan of Alg. 3 is the one step that looks across the cut: the 3x3x3 local
maximum of a cell on the first or last fine-v row of a rank needs the neighbouring rank's
border row.  So each rank sends its first and last fine-v rows to its neighbours (the only
map data that crosses between GPUs), scans its rows with those halo rows as neighbours
(detect_peaks_add), keeps its top K (detect_peaks_end), and the ranks all-gather these
lists; detect_merge of the gathered lists is the top K of the whole grid, identical on
every rank to the single-GPU result.

The functions take a torch.distributed process group: NCCL with CUDA tensors on GPUs, or
gloo with CPU tensors (the host logic is tested that way)."""
from __future__ import annotations

import torch
import torch.distributed as dist


def coarse_rows(nvc: int, world: int, rank: int):
    """[i0, i1): the contiguous block of coarse-v rows of rank `rank`, the first nvc % world
    ranks taking one row more.  Every rank gets at least one row (world <= nvc)."""
    if not (0 < world <= nvc) or not (0 <= rank < world):
        raise ValueError(f"{world} ranks over {nvc} coarse rows")
    base, extra = divmod(nvc, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def exchange_halos(first_row, last_row, above, below, group=None):
    """Send this rank's first row to rank - 1 and its last row to rank + 1; receive rank - 1's
    last row into `above` and rank + 1's first row into `below` (either is ignored at the
    ends of the grid).  All four tensors have the shape of one fine-v row."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, first_row.contiguous(), rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, above, rank - 1, group))
    if rank + 1 < world:
        ops.append(dist.P2POp(dist.isend, last_row.contiguous(), rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, below, rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def gather_detections(out, n_out, group=None):
    """All-gather every rank's detection list (a uint8 buffer of K records) and total into
    (lists: uint8 [world * len(out)], totals: int32 [world]), rank order."""
    world = dist.get_world_size(group)
    lists = [torch.empty_like(out) for _ in range(world)]
    totals = [torch.empty_like(n_out) for _ in range(world)]
    dist.all_gather(lists, out.contiguous(), group=group)
    dist.all_gather(totals, n_out.reshape(1).contiguous(), group=group)
    return torch.cat(lists), torch.cat(totals).reshape(world)


def sharded_dsgrft_detect(radar, echo, grid, precision, cfar, K, group=None):
    """The top K detections of the whole DS grid, computed with the coarse-v rows split over
    the ranks of `group` (one GPU each, echo replicated).  Returns (out, n_out) on every rank,
    equal to dsgrft_detect on one GPU."""
    from . import (detect_merge, detect_peaks_add, detect_peaks_begin, detect_peaks_end,
                   dsgrft_fine_dfm)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    nvc, nac, Fv = int(grid.vc.count), int(grid.ac.count), int(grid.Fv)
    na, nr0 = nac * int(grid.Fa), int(grid.r0_count)
    i0, i1 = coarse_rows(nvc, world, rank)
    rows = (i1 - i0) * Fv
    # this rank's rows with a halo row on either side
    P = torch.empty((rows + 2, na, nr0), dtype=torch.float32, device=echo.device)
    dsgrft_fine_dfm(radar, None, echo, grid, i0 * nac, (i1 - i0) * nac, precision, None, P[1:rows + 1])
    exchange_halos(P[1], P[rows], P[0], P[rows + 1], group)
    lo = 1 if rank == 0 else 0                       # the grid's ends have no halo row
    hi = rows + 2 if rank + 1 < world else rows + 1
    detect_peaks_begin()
    detect_peaks_add(P[lo:hi], 1 - lo, 1 - lo + rows, i0 * Fv - (1 - lo), cfar)
    out, n_out = detect_peaks_end(na, nr0, K, axes=grid.plain_equivalent(), dr_m=radar.dr_m, device=echo.device)
    lists, totals = gather_detections(out, n_out, group)
    return detect_merge(lists, totals, K, K)
