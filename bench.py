"""Benchmark of the DS-GRFT hot path on GB300 (hypothesis*pulse MAC/s).

One step = one pass of the whole DS-GRFT path over one CPI of the 2^30-hypothesis
workload (M=512 pulses x N=4096 bins, f_c 1.5 GHz, PRF 1 kHz; coarse 4096 r0 x 32 v x 8 a,
fine 64 x 16): FP64 tables, fused coarse-RM gather + fine-DFM tensor-core contraction +
|Y|^2 epilogue, CA-CFAR + top-K with the estimate map.  Plain GRFT over the same
hypotheses is timed beside it (the DS speedup), and the FP64 oracle is timed on a bounded
sample on the host cores.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp16x2]
"""
from __future__ import annotations

import argparse
import atexit
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DS-GRFT vs plain GRFT hypothesis·pulse MACs/s, 1 GB300, ≤2e-3 rel peak err"
UNIT = "hyp*pulse/s"
WORKLOAD = "DS-GRFT, M=512 x N=4096 complex64, 4096 r0 x (32x64) v x (8x16) a = 2^30 hypotheses"
FLOP_PER_HYP_PULSE = 8          # one complex multiply-add
ACC_ROWS = 512                  # random (v, a) rows of the accuracy check (every r0 bin)
# ncu dram__bytes_read.sum + dram__bytes_write.sum of the contraction kernel on the first 16
# coarse cells, scaled by 16 to one launch of this workload (all 256 cells in one launch),
# per precision.  None until a capture of the current kernel exists.
DRAM_TRAFFIC_PER_LAUNCH = {"fp16x2": 16 * (269.672960e6 + 219.864064e6)}   # k_ds_pair<3, 2, 224>
PRODUCTS_PER_MAC = {"bf16x3": 3, "fp16x3": 3, "fp16x2": 2, "fp16x1": 1, "fp32": 1}
def pair_bn(slots):
    """Tile width (B rows, two per slot) the pair form's contraction takes: of 256, 224 and 192
    the one with the fewest tiles, then the fewest columns."""
    best, best_tiles = 256, -(-slots // 128)
    best_cols = best_tiles * 256
    for bn in (224, 192):
        tiles = -(-slots // (bn // 2))
        if tiles < best_tiles or (tiles == best_tiles and tiles * bn < best_cols):
            best, best_tiles, best_cols = bn, tiles, tiles * bn
    return best


def executed_per_algorithmic(precision, Fv, Fa):
    """Tensor FLOP the contraction executes per algorithmic FLOP (8 per hypothesis-pulse).  The
    pair form (P = 2 grids) contracts each slot of mirrored hypotheses (every hypothesis once,
    with its mirror where it has one: Fa + Fv - 1 + ceil((Fv - 1)(Fa - 1) / 2) slots, padded to
    whole tiles of pair_bn / 2 slots) as four real MACs per pulse and product, i.e. 8 FLOP per
    slot-pulse and product."""
    if precision == "fp32":
        return 1.0
    if os.environ.get("DSGRFT_PAIR", "1").startswith("0"):      # the 4M form
        return float(PRODUCTS_PER_MAC[precision])
    slots = Fa + (Fv - 1) + ((Fv - 1) * (Fa - 1) + 1) // 2
    half = pair_bn(slots) // 2
    spad = -(-slots // half) * half
    return PRODUCTS_PER_MAC[precision] * spad / float(Fv * Fa)


# arithmetic type of the contraction's operands (accumulation is FP32 in every mode)
DTYPE = {"bf16x3": "bf16", "fp16x3": "f16", "fp16x2": "f16", "fp16x1": "f16", "fp32": "f32"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms by a reader thread.  The
    sampler starts before the warm-up (nvidia-smi takes a while to print its first line);
    mark() brackets the timed region and summary() keeps the samples taken inside it (the
    first one after it if the region is shorter than the period)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.samples = []              # (monotonic time, line)
        self.t0 = self.t1 = None
        self.thread = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.monotonic(), line))

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if self.proc is None or self.proc.poll() is not None:
            return
        time.sleep(0.15)               # one more period, for a region shorter than it
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [l for t, l in self.samples if self.t0 is not None and self.t0 <= t <= self.t1]
        if not lines and self.t0 is not None:
            after = [l for t, l in self.samples if t > self.t1]
            lines = after[:1]
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw)}


def _cpu_oracle_sample(sc, s, target_s: float, warm_rows: int = 8, threads: int = 0):
    """Time the FP64 oracle on (cell, fine) rows of the DS grid, every r0 and pulse, on
    `threads` host threads (0: all)."""
    import oracle
    ds = sc.ds
    nthreads = threads if threads > 0 else oracle.num_threads()
    rng = np.random.default_rng(0)
    def rows(n):
        return rng.integers(0, ds.n_cells, n), rng.integers(0, ds.n_fine, n)
    c, f = rows(max(warm_rows, nthreads))
    t0 = time.perf_counter()
    oracle.dsgrft_rows(sc.radar, s, ds, c, f, nthreads=threads)
    rate = c.size / (time.perf_counter() - t0)
    n = int(max(nthreads, min(200000, rate * target_s)))
    c, f = rows(n)
    t0 = time.perf_counter()
    oracle.dsgrft_rows(sc.radar, s, ds, c, f, nthreads=threads)
    dt = time.perf_counter() - t0
    units = n * ds.r0_count * sc.radar.M
    return units / dt, nthreads, n, dt


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample of the same workload."""
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sc = synth.ds_m512()
    s = synth.make_echo(sc.radar, sc.targets, sc.seed)
    for _ in range(args.warmup):
        _cpu_oracle_sample(sc, s, target_s=1.0)
    vals, cores, nrows, tot = [], 0, 0, 0.0
    step_s = min(args.ref_step_s, args.ref_total_s / max(1, args.steps))   # the whole run stays bounded
    for _ in range(args.steps):
        v, cores, n, dt = _cpu_oracle_sample(sc, s, target_s=step_s)
        vals.append(v)
        nrows += n
        tot += dt
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "oracle rows"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{nrows} (cell, fine) rows x 4096 r0 x 512 pulses over {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def residual_migration(radar, ds) -> dict:
    """The dual-scale approximation's residual range migration (eq. Residual_RM_DeltaR): a
    fine offset moves at most (dv_c T + da_c T^2 / 2) / 2 over the CPI, T = M / PRF; the
    coarse bins stay valid for the fine hypotheses while that is at most dr / 2."""
    T = radar.M / radar.prf_hz
    res = 0.5 * (ds.vc.step * T + 0.5 * ds.ac.step * T * T)
    return {"residual_m": res, "half_bin_m": 0.5 * radar.dr_m, "rm_bound_ok": bool(res <= 0.5 * radar.dr_m)}


# ---------------------------------------------------------------- multi-rank plumbing
# One process per GPU; every rank processes its own CPI (weak scaling) and nothing crosses
# ranks on the data path: the only collectives are the timing barrier and the max below.
def rank_layout():
    """(world, rank, local rank) from the launcher's environment; (1, 0, 0) without one."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks (the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_per_step: float) -> float:
    """Whole-job throughput: world ranks each process units_per_rank per step."""
    return world * units_per_rank / seconds_per_step


def _timed(fn, reps, stream):
    """Average CUDA-event time (ms) of fn() over reps calls after one untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _contract_roofline(g, units, fn, steps, stream):
    """Run fn `steps` times with the library's per-kernel events on and return the roofline of
    the tensor-core contraction over those calls: algorithmic FLOP (8 per hypothesis-pulse of
    `units` per call) over the contraction kernel's own time, against the measured burst
    BF16 rate (dense FP16 is the same rate), plus the other kernels' shares."""
    torch = sys.modules["torch"]
    torch.cuda.synchronize()
    g.grft_timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    kt = {k: g.grft_timing_get(k) for k in ("tables", "split", "contract", "cfar", "topk")}
    g.grft_timing(False)
    call_ms = a.elapsed_time(b) / steps
    n_c, ms_c = kt["contract"]
    peak = _peaks()[0].get("bf16_tflops", 1930.4)
    r = {"call_ms": call_ms, "kernels_ms_per_call": {k: v[1] / steps for k, v in kt.items() if v[0] > 0}}
    if n_c > 0 and ms_c > 0:
        ach = FLOP_PER_HYP_PULSE * units * steps / (1e-3 * ms_c) / 1e12
        r["roofline"] = {"bound": "tensor", "kernel": "k_ds_tc (all launches of the call)", "achieved": ach,
                         "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "launches_per_call": n_c / steps,
                         "peak_source": "measured bf16_tflops (burst); dense FP16 and BF16 rates are equal"}
    return r


def run_suite(args):
    """The other workloads of the method, one JSON line: the M=2048 x N=8192 precision case
    (one coarse-v row of cells per call, both split precisions, sampled error against the
    oracle; and the whole 3.4e10-hypothesis grid with streamed detection), 64 uneven CPIs
    with every range bin (groups of batched launches plus detection, one CUDA graph) and
    with 1024 range bins of interest per CPI (one graph-captured batched call), the
    differentiation pipeline at M=1024 x N=4096 (forward, top-1000 CFAR,
    adjoint, 20 refinement steps), the FFT form of the fine stage and the frequency-domain
    coarse stage against their dense / gather forms, and the keystone branch (DS-KT-MFP)
    over its 1.88e9-hypothesis grid."""
    import torch
    import paper_2403_06788_gb300 as g
    import synth
    dev = torch.device("cuda", 0)
    g.load()
    stream = torch.cuda.current_stream()
    out = {}

    # ------------------------------------------------ precision workload, one coarse-v row
    sc = synth.ds_precision_m2048()
    R, ds = sc.radar, sc.ds
    s = synth.make_echo(R, sc.targets, sc.seed)
    echo = torch.from_numpy(s).to(dev)
    t = max(sc.targets, key=lambda t: abs(t.amp))
    pg = ds.plain_equivalent()
    i_row = min(int((t.v - pg.v.start) // ds.vc.step), ds.vc.count - 1)
    cb, cc = i_row * ds.ac.count, ds.ac.count
    nv, na = ds.Fv, ds.ac.count * ds.Fa
    Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device=dev)
    units = cc * ds.n_fine * ds.r0_count * R.M
    prec = {}
    rng = np.random.default_rng(0)
    vloc, af = rng.integers(0, nv, 6), rng.integers(0, na, 6)
    Yo = None
    if not args.no_cpu:
        import oracle
        from oracle.wrap import ds_rows_of_canonical
        cell, fine = ds_rows_of_canonical(ds, np.asarray(vloc) + i_row * ds.Fv, np.asarray(af))
        Yo = oracle.dsgrft_rows(R, s, ds, cell, fine)
    for p in ("bf16x3", "fp16x3"):
        ms = _timed(lambda: g.dsgrft_fine_dfm(R, None, echo, ds, cb, cc, p, Y, None), 3, stream)
        err = None
        if Yo is not None:
            Yg = Y[torch.as_tensor(vloc, device=dev), torch.as_tensor(af, device=dev)].cpu().numpy()
            err = float(np.abs(Yg - Yo).max() / np.abs(Yo).max())
        prec[p] = {"ms_per_call": ms, "value": units / (1e-3 * ms), "max_rel_peak_err_sampled": err}
    out["precision_m2048"] = {"workload": "DS-GRFT M=2048 x N=8192, coarse 32 x 8, fine 256 x 64; one call = "
                                          "one coarse-v row (8 cells, 2.2e12 hypothesis-pulses, Y written)",
                              "unit": UNIT, "full_grid_calls": ds.vc.count,
                              "range_migration": residual_migration(R, ds), **prec}
    del Y, echo
    torch.cuda.empty_cache()

    # ------------------------------------------------ precision workload, whole grid, streamed detection
    # every one of the 3.4e10 hypotheses: dsgrft_detect computes one coarse-v row of cells at a
    # time into a slab buffer and scans it (halo rows from its neighbours), top 1000 overall
    sc = synth.ds_precision_m2048()
    R, ds = sc.radar, sc.ds
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).to(dev)
    cf = synth.CFAR(2, 16, 1e-6)
    K = 1000
    det = torch.zeros(K * g._abi.DET_BYTES, dtype=torch.uint8, device=dev)
    nout = torch.zeros(1, dtype=torch.int32, device=dev)
    units = ds.n_cells * ds.n_fine * ds.r0_count * R.M
    full = {}
    for p in ("fp16x2", "bf16x3"):
        run = lambda: g.dsgrft_detect(R, echo, ds, p, cf, K, out=det, n_out=nout)
        run()
        r = _contract_roofline(g, units, run, 2, stream)
        dets, total = g.decode_detections(det, nout, K)
        pgd = ds.plain_equivalent()
        found = 0
        for t in sc.targets:        # a detection within one cell of the target on every axis
            near = (np.abs(dets["r0_m"] / R.dr_m - t.r0_bins) <= 1.5) & \
                (np.abs(dets["v"] - t.v) <= 1.5 * pgd.v.step) & (np.abs(dets["a"] - t.a) <= 1.5 * pgd.a.step)
            found += int(near.any())
        full[p] = dict(r, value=units / (1e-3 * r["call_ms"]), detections_total=total,
                       targets_detected=f"{found} of {len(sc.targets)}", status=g.grft_sync_status())
    out["precision_m2048_full"] = {
        "workload": "DS-GRFT M=2048 x N=8192, coarse 32 x 8, fine 256 x 64, every r0 bin: 3.4e10 hypotheses "
                    "(7.0e13 hypothesis-pulses) per call, streamed one coarse-v row of cells at a time into a "
                    "slab buffer (4.3 GB) with CA-CFAR + local maximum + top 1000 over the whole grid; the "
                    "137 GB power map is never held",
        "unit": UNIT, "hypotheses": ds.n_cells * ds.n_fine * ds.r0_count, "pulses": R.M,
        "range_migration": residual_migration(R, ds), **full}
    del echo, det
    torch.cuda.empty_cache()

    # ------------------------------------------------ 64 CPIs, every r0 bin, one captured graph
    # the 64 power maps (about 300 GB) do not fit at once: CPIs go in groups whose maps fit a
    # 96 GiB buffer, each group one batched launch followed by a top-64 detection per CPI; the
    # whole sequence is one CUDA graph
    cpis = synth.ds_batch(n_cpi=64)
    grid = cpis[0].ds
    nvb, nab = grid.vc.count * grid.Fv, grid.ac.count * grid.Fa
    budget = 96 << 30
    Kc = 64
    echoes = [torch.from_numpy(synth.make_echo(c.radar, c.targets, c.seed)).to(dev) for c in cpis]
    groups, cur, used = [], [], 0
    for k, c in enumerate(cpis):
        nb = nvb * nab * c.radar.N * 4
        if cur and used + nb > budget:
            groups.append(cur)
            cur, used = [], 0
        cur.append((k, used))
        used += nb
    groups.append(cur)
    pbuf = torch.empty(budget // 4, dtype=torch.float32, device=dev)
    dets_all = torch.zeros((len(cpis), Kc * g._abi.DET_BYTES), dtype=torch.uint8, device=dev)
    n_all = torch.zeros((len(cpis), 1), dtype=torch.int32, device=dev)
    units = sum(nvb * nab * c.radar.N * c.radar.M for c in cpis)

    def run_all(prec):
        for grp in groups:
            items = []
            for k, off in grp:
                N = cpis[k].radar.N
                P = pbuf[off // 4: off // 4 + nvb * nab * N].view(nvb, nab, N)
                items.append({"echo": echoes[k], "P": P, "Y": None, "r0_begin": 0, "r0_count": N})
            g.dsgrft_fine_dfm_batched(cpis[0].radar, grid, items, prec)
            for (k, off), it in zip(grp, items):
                g.detect_peaks(it["P"], cf, Kc, out=dets_all[k], n_out=n_all[k])

    batch_full = {}
    for p in ("fp16x2",):
        run_all(p)                                   # sizes the workspaces, tunes the tiles
        r = _contract_roofline(g, units, lambda: run_all(p), 1, stream)
        side = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            run_all(p)
        ms = _timed(graph.replay, 2, stream)
        tot = n_all.cpu().numpy().ravel()
        batch_full[p] = dict(r, graph_ms_per_call=ms, value=units / (1e-3 * ms), groups=len(groups),
                             detections_per_cpi_min=int(tot.min()), detections_per_cpi_max=int(tot.max()),
                             status=g.grft_sync_status())
        del graph
    out["batch_64_full"] = {
        "workload": "64 CPIs, M ~ U{256..2048}, N ~ U{1024..8192}, coarse 32 x 8, fine 64 x 16, every r0 bin "
                    "of every CPI (%.3g hypothesis-pulses); groups of CPIs whose maps fit 96 GiB, one batched "
                    "launch and a top-64 CA-CFAR detection per CPI each, the whole sequence one CUDA graph" % units,
        "unit": UNIT, "hypothesis_pulses": units, **batch_full}
    del pbuf, echoes, dets_all
    torch.cuda.empty_cache()

    # ------------------------------------------------ 64 uneven CPIs, one captured batched call
    cpis = synth.ds_batch(n_cpi=64)
    grid = cpis[0].ds
    nvb, nab = grid.vc.count * grid.Fv, grid.ac.count * grid.Fa
    batch, units = [], 0
    for sc in cpis:
        N = sc.radar.N
        r0c = min(1024, N)
        e = torch.from_numpy(synth.make_echo(sc.radar, sc.targets, sc.seed)).to(dev)
        P = torch.empty((nvb, nab, r0c), device=dev)
        batch.append({"echo": e, "P": P, "Y": None, "r0_begin": (N - r0c) // 2, "r0_count": r0c})
        units += nvb * nab * r0c * sc.radar.M
    g.dsgrft_fine_dfm_batched(cpis[0].radar, grid, batch, "bf16x3")         # sizes the workspace, tunes
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        g.dsgrft_fine_dfm_batched(cpis[0].radar, grid, batch, "bf16x3")
    ms = _timed(graph.replay, 3, stream)
    out["batch_64"] = {"workload": "64 CPIs, M ~ U{256..2048}, N ~ U{1024..8192}, coarse 32 x 8, fine 64 x 16, "
                                   "1024 range bins of interest per CPI, one graph-captured batched call",
                       "unit": UNIT, "ms_per_call": ms, "value": units / (1e-3 * ms),
                       "status": g.grft_sync_status()}
    del batch, graph
    torch.cuda.empty_cache()

    # ------------------------------------------------ differentiation pipeline
    sc = synth.ds_adjoint_m1024()
    R, ds = sc.radar, sc.ds
    pg = ds.plain_equivalent()
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).to(dev)
    P = torch.empty((ds.vc.count * ds.Fv, ds.ac.count * ds.Fa, ds.r0_count), device=dev)
    det = torch.zeros(1000 * g._abi.DET_BYTES, dtype=torch.uint8, device=dev)
    nout = torch.zeros(1, dtype=torch.int32, device=dev)
    cfar = synth.CFAR(2, 16, 1e-6)
    units = ds.n_cells * ds.n_fine * ds.r0_count * R.M
    ms_fwd = _timed(lambda: g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.n_cells, "bf16x3", None, P), 3, stream)
    ms_det = _timed(lambda: g.detect_peaks(P, cfar, 1000, axes=pg, dr_m=R.dr_m, out=det, n_out=nout), 3, stream)
    dets, total = g.decode_detections(det, nout, 1000)
    th0 = torch.from_numpy(np.stack([dets["r0_m"], dets["v"], dets["a"]], axis=1).astype(np.float64)).to(dev)
    K = th0.shape[0]
    gt = torch.empty((K, 3), dtype=torch.float64, device=dev)
    ms_adj = _timed(lambda: g.dsgrft_backward(R, echo, th0, 1, grad_theta=gt), 3, stream)
    cellw = [R.dr_m, pg.v.step, pg.a.step]
    Pr = torch.empty(K, device=dev)
    th = th0.clone()

    def refine():
        th.copy_(th0)
        g.dsgrft_refine(R, echo, th, cellw, 20, 1, Pr)
    ms_ref = _timed(refine, 3, stream)
    out["differentiation_m1024"] = {
        "workload": "DS-GRFT M=1024 x N=4096 (2^30 hypotheses), top-1000 CA-CFAR, adjoint at the detections, "
                    "20 ascent steps (linear gather)",
        "range_migration": residual_migration(R, ds),
        "detections": int(K), "forward_ms": ms_fwd, "forward_value": units / (1e-3 * ms_fwd), "unit": UNIT,
        "detect_ms": ms_det, "adjoint_ms": ms_adj, "refine_20_steps_ms": ms_ref,
        "status": g.grft_sync_status()}
    del P, echo
    torch.cuda.empty_cache()

    out.update(measure_forms(0, 3, 1))
    out["keystone_m512"] = measure_kt(rows=0, steps=3, warmup=1)
    out["p3_m512"] = {p: measure_p3(3, 1, p) for p in ("fp16x2", "bf16x3")}
    print(json.dumps({"suite": out}))
    return 0


def measure_forms(cells=0, steps=3, warmup=1):
    """The paper's own forms of the two stages on the M=512 x N=4096 echo: the FFT form of
    the fine stage (Alg. 2; fine velocity step one bin of a 512-point transform, 96 x 16 fine
    hypotheses per cell) against the dense split-BF16 contraction of the same hypotheses, and
    the frequency-domain coarse stage (Alg. 1) against the time-domain TMA gather, into Z.
    cells > 0: the first `cells` coarse cells only (a profiling case); else all 256 for the
    fine stage and 32 for the coarse stage (Z of 32 cells = 537 MB)."""
    import torch
    import paper_2403_06788_gb300 as g
    import synth
    dev = torch.device("cuda", 0)
    g.load()
    stream = torch.cuda.current_stream()
    sc = synth.ds_m512()
    R = sc.radar
    L, Fv = 512, 96                                   # fine velocity step = one bin of 512
    vstep = R.wavelength * R.prf_hz * Fv / (2 * L)
    ds = synth.DSGrid(0, R.N, synth.Axis(-300.0 + vstep / 2, vstep, 32), sc.ds.ac, Fv, sc.ds.Fa)
    nc = ds.n_cells if cells <= 0 else min(cells, ds.n_cells)
    nrow = (nc + ds.ac.count - 1) // ds.ac.count
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).to(dev)
    P = torch.empty((nrow * Fv, ds.ac.count * ds.Fa, ds.r0_count), device=dev)
    units = nc * ds.n_fine * ds.r0_count * R.M

    def timed(fn):
        for _ in range(max(warmup, 1)):
            fn()
        return _timed(fn, steps, stream)
    ms_fft = timed(lambda: g.dsgrft_fine_dfm_fft(R, echo, ds, 0, nc, None, P))
    ms_dense = timed(lambda: g.dsgrft_fine_dfm(R, None, echo, ds, 0, nc, "bf16x3", None, P))
    del P
    torch.cuda.empty_cache()
    dsz = sc.ds
    ncz = 32 if cells <= 0 else min(cells, 32)
    Z = torch.empty((ncz, R.M, dsz.r0_count), dtype=torch.complex64, device=dev)
    ms_fd = timed(lambda: g.dsgrft_coarse_rm_fd(R, echo, dsz, 0, ncz, Z))
    ms_td = timed(lambda: g.dsgrft_coarse_rm(R, echo, dsz, 0, ncz, Z))
    del Z, echo
    torch.cuda.empty_cache()
    return {
        "coarse_stage_m512": {
            "workload": f"coarse range-migration correction of {ncz} cells x 512 pulses x 4096 bins into Z "
                        "(complex64)",
            "frequency_domain_ms": ms_fd, "time_domain_gather_ms": ms_td,
            "frequency_domain_rows_per_s": ncz * R.M / (1e-3 * ms_fd)},
        "fft_form_m512": {
            "workload": f"DS-GRFT M=512 x N=4096, {nc} coarse cells (of 32 x 8), fine 96 x 16 (fine velocity step = "
                        "one bin of a 512-point transform), P written",
            "hypotheses": nc * ds.n_fine * ds.r0_count,
            "unit": UNIT, "fft_ms": ms_fft, "fft_value": units / (1e-3 * ms_fft),
            "dense_bf16x3_ms": ms_dense, "dense_value": units / (1e-3 * ms_dense),
            "status": g.grft_sync_status()}}


def run_forms(args):
    print(json.dumps({"forms": measure_forms(args.cells, args.steps, args.warmup)}))
    return 0


def measure_kt(rows=0, steps=3, warmup=3):
    """The keystone branch (DS-KT-MFP, Alg. 4) on the ds_m512 echo: dskt_mfp over q in
    [-3, 3] (rows > 0: the first `rows` folding factors only, a profiling case) x 8 coarse a
    cells, 512 baseband v bins x 16 fine a per cell, 4096 r0, P written (7.5 GB, larger than
    L2), then top-1000 CA-CFAR.  CUDA events around `steps` steps after `warmup`; per-kernel
    times from the library's own events; the fine-stage kernel's algorithmic bytes and FLOP."""
    import dataclasses
    import torch
    import paper_2403_06788_gb300 as g
    import synth
    dev = torch.device("cuda", 0)
    g.load()
    stream = torch.cuda.current_stream()
    sc = synth.dskt_m512()
    R, ds = sc.radar, sc.ds
    if rows > 0:
        ds = dataclasses.replace(ds, vc=synth.Axis(ds.vc.start, ds.vc.step, min(rows, ds.vc.count)))
    pgk = ds.plain_equivalent()
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).to(dev)
    P = torch.empty((ds.vc.count * ds.Fv, ds.ac.count * ds.Fa, ds.r0_count), device=dev)
    det = torch.zeros(1000 * g._abi.DET_BYTES, dtype=torch.uint8, device=dev)
    nout = torch.zeros(1, dtype=torch.int32, device=dev)
    cfar = synth.CFAR(2, 16, 1e-6)
    for _ in range(max(warmup, 1)):
        g.dskt_mfp(R, echo, ds, None, P)
        g.detect_peaks(P, cfar, 1000, axes=pgk, dr_m=R.dr_m, out=det, n_out=nout)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    g.grft_timing(True)
    for e0, e1, e2 in ev:
        e0.record(stream)
        g.dskt_mfp(R, echo, ds, None, P)
        e1.record(stream)
        g.detect_peaks(P, cfar, 1000, axes=pgk, dr_m=R.dr_m, out=det, n_out=nout)
        e2.record(stream)
    torch.cuda.synchronize()
    kt = {k: g.grft_timing_get(k) for k in ("tables", "keystone", "coarse_rm", "contract_fft", "cfar", "topk")}
    g.grft_timing(False)
    map_ms = sum(a.elapsed_time(b) for a, b, c in ev) / steps
    det_ms = sum(b.elapsed_time(c) for a, b, c in ev) / steps
    dets, total = g.decode_detections(det, nout, 1000)
    found = 0
    for t in sc.targets:
        found += int(((np.abs(dets["r0_m"] / R.dr_m - t.r0_bins) <= 1.0) & (np.abs(dets["v"] - t.v) <= 2 * pgk.v.step)
                      & (np.abs(dets["a"] - t.a) <= 2 * pgk.a.step)).any())
    units = ds.n_hyp * R.M
    z_bytes = ds.n_cells * R.M * ds.r0_count * 8
    L = ds.Fv
    fine_ms = kt["contract_fft"][1] / max(kt["contract_fft"][0], 1)
    fine_bytes = z_bytes + ds.n_hyp * 4
    fine_flop = ds.n_cells * ds.r0_count * ds.Fa * (10.0 * (L // 2) * int(math.log2(L)) + 6.0 * L)
    res = {
        "workload": f"DS-KT-MFP on the ds_m512 echo (M=512 x N=4096): keystone transform, q in "
                    f"[-3, {ds.vc.count - 4}] x 8 coarse a cells (H_KT,RM coarse stage), 512 baseband v bins "
                    f"x 16 fine a per cell (FFT form), 4096 r0: {ds.n_hyp:.3g} hypotheses, P written; then "
                    "top-1000 CA-CFAR",
        "unit": UNIT, "steps": steps, "map_ms": map_ms, "detect_ms": det_ms, "value": units / (1e-3 * map_ms),
        "step_value": units / (1e-3 * (map_ms + det_ms)),
        "kernels_ms_per_step": {k: v[1] / steps for k, v in kt.items()},
        "fine_stage": {"bytes_per_launch": fine_bytes, "flop_per_launch": fine_flop, "ms_per_launch": fine_ms,
                       "achieved_gbs": fine_bytes / (1e-3 * fine_ms) / 1e9,
                       "achieved_tflops": fine_flop / (1e-3 * fine_ms) / 1e12},
        "targets_found": f"{found}/{len(sc.targets)}", "detections": int(total),
        "status": g.grft_sync_status()}
    del P, echo
    torch.cuda.empty_cache()
    return res


def measure_p3(steps=3, warmup=1, precision="bf16x3"):
    """DS-GRFT with the acceleration rate (P = 3) on the ds3_m512 workload (M=512 x N=4096,
    coarse 8 v x 8 a x 4 b, fine 64 x 8 x 4: 2.1e9 hypotheses), P written (8.6 GB, larger
    than L2): CUDA events around `steps` calls after `warmup`."""
    import torch
    import paper_2403_06788_gb300 as g
    import synth
    dev = torch.device("cuda", 0)
    g.load()
    stream = torch.cuda.current_stream()
    sc = synth.ds3_m512()
    R, g3 = sc.radar, sc.ds3
    echo = torch.from_numpy(synth.make_echo(R, sc.targets, sc.seed)).to(dev)
    shape = (g3.vc.count * g3.Fv, g3.ac.count * g3.Fa, g3.bc.count * g3.Fb, g3.r0_count)
    P = torch.empty(shape, device=dev)
    ncell = g3.vc.count * g3.ac.count * g3.bc.count
    run = lambda: g.dsgrft3_fine_dfm(R, echo, g3, 0, ncell, precision, None, P)
    for _ in range(max(warmup, 1)):
        run()
    ms = _timed(run, steps, stream)
    units = g3.n_hyp * R.M
    res = {"workload": "DS-GRFT P=3 (acceleration rate), M=512 x N=4096, coarse 8 v x 8 a x 4 b, fine 64 x 8 x 4, "
                       "4096 r0 = 2.1e9 hypotheses, P written", "precision": precision, "unit": UNIT,
           "ms_per_call": ms, "value": units / (1e-3 * ms), "status": g.grft_sync_status()}
    del P, echo
    torch.cuda.empty_cache()
    return res


def run_kt(args):
    print(json.dumps({"keystone": measure_kt(args.kt_rows, args.steps, args.warmup)}))
    return 0


def pd_hit(vi, ai, n0s, j, k, n0) -> bool:
    """A Monte-Carlo trial detects when some detection (vi, ai, n0s) lies within one cell of
    the truth (j, k, n0) on every axis."""
    vi, ai, n0s = (np.asarray(x).astype(np.int64) for x in (vi, ai, n0s))
    return bool(((np.abs(vi - j) <= 1) & (np.abs(ai - k) <= 1) & (np.abs(n0s - n0) <= 1)).any())


def run_pd(args):
    """Detection probability against SNR for plain GRFT, DS-GRFT (time-domain coarse gather
    and, as the paper computes it, frequency-domain coarse stage) and DS-KT-MFP (the paper's
    Monte-Carlo comparison, Sec. VI): M=256 x N=512, one target per trial at a random
    on-grid (r0, v, a), CN(0,1) noise, the fixed LRT threshold -M ln(Pfa) on |Y|^2 with the
    3x3x3 local maximum; a trial detects when a detection lies within one cell of the truth
    on every axis (pd_hit).  The keystone grid (q in [-1, 1], 256 baseband bins of V_a / 256
    = the DS-GRFT fine velocity step) contains every DS-GRFT hypothesis.  Trial inputs come
    from synth.pd_trial (one seed per trial).  One JSON line."""
    import torch
    import paper_2403_06788_gb300 as g
    import synth
    dev = torch.device("cuda", 0)
    g.load()
    R, ds, ktg, cf = synth.pd_setup()
    pg = ds.plain_equivalent()
    nv, na = pg.v.count, pg.a.count
    K = 64
    P = torch.empty((nv, na, R.N), device=dev)
    kpg = ktg.plain_equivalent()
    kv_off = int(round((pg.v.start - kpg.v.start) / kpg.v.step))   # same velocity lattice
    assert abs(kpg.v.step - pg.v.step) < 1e-12 and abs(kpg.v.start + kv_off * kpg.v.step - pg.v.start) < 1e-9
    Pk = torch.empty((kpg.v.count, na, R.N), device=dev)
    Zfd = torch.empty((ds.n_cells, R.M, R.N), dtype=torch.complex64, device=dev)
    snrs = [float(x) for x in args.pd_snr.split(",")]
    res = {}
    for snr in snrs:
        hits = {"grft": 0, "dsgrft": 0, "dsgrft_fd": 0, "dsktmfp": 0}
        for trial in range(args.pd_trials):
            j, k, n0, s_np = synth.pd_trial(R, pg, snr, trial)
            echo = torch.from_numpy(s_np).to(dev)
            for name in ("grft", "dsgrft", "dsgrft_fd", "dsktmfp"):
                jt = j
                if name == "grft":
                    g.grft_plain(R, echo, pg, None, P)
                    out, n = g.detect_peaks(P, cf, K)
                elif name == "dsgrft":
                    g.dsgrft_fine_dfm(R, None, echo, ds, 0, ds.n_cells, "bf16x3", None, P)
                    out, n = g.detect_peaks(P, cf, K)
                elif name == "dsgrft_fd":               # the paper's form: mGIFT in range frequency
                    g.dsgrft_coarse_rm_fd(R, echo, ds, 0, ds.n_cells, Zfd)
                    g.dsgrft_fine_dfm(R, Zfd, echo, ds, 0, ds.n_cells, "bf16x3", None, P)
                    out, n = g.detect_peaks(P, cf, K)
                else:
                    g.dskt_mfp(R, echo, ktg, None, Pk)
                    out, n = g.detect_peaks(Pk, cf, K)
                    jt = j + kv_off
                dets, _ = g.decode_detections(out, n, K)
                hits[name] += int(pd_hit(dets["vi"], dets["ai"], dets["n0"], jt, k, n0))
        res[f"{snr:g}"] = {name: hits[name] / args.pd_trials for name in hits}
    print(json.dumps({"pd": {
        "workload": "M=256 x N=512, f_c 1.5 GHz, PRF 1 kHz; GRFT / DS-GRFT (time-domain gather; dsgrft_fd: "
                    "frequency-domain coarse stage): coarse 8 x 2, fine 64 x 8 (512 v x 16 a "
                    "x 512 r0); DS-KT-MFP: q in [-1, 1] x 2 a cells, 256 baseband v x 8 a (768 v x 16 a x 512 r0, "
                    "same lattice); one on-grid target per trial, CN(0,1) noise, fixed threshold -M ln(1e-6) + "
                    "local maximum",
        "snr_db_per_sample": snrs, "trials_per_snr": args.pd_trials, "pd": res,
        "range_migration": residual_migration(R, ds), "status": g.grft_sync_status()}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)  # about 0.5 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x2", choices=["bf16x3", "fp16x3", "fp16x2", "fp16x1", "fp32"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--ref-total-s", type=float, default=120.0)
    ap.add_argument("--topk", type=int, default=1000)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline and accuracy check")
    ap.add_argument("--cells", type=int, default=0,
                    help="restrict to the first N coarse cells (small profiling case; not a bench line)")
    ap.add_argument("--e2e-steps", type=int, default=0)
    ap.add_argument("--pd", action="store_true",
                    help="Monte-Carlo detection probability of plain GRFT and DS-GRFT against SNR (one JSON line)")
    ap.add_argument("--pd-trials", type=int, default=100)
    ap.add_argument("--pd-snr", default="-18,-15,-13,-11,-9,-6")
    ap.add_argument("--suite", action="store_true",
                    help="time the precision, batching and differentiation workloads (one JSON line)")
    ap.add_argument("--forms", action="store_true",
                    help="time the FFT-form fine stage and the frequency-domain coarse stage against the dense "
                         "and gather forms (one JSON line; --cells N: the first N cells)")
    ap.add_argument("--other-precisions", default="bf16x3,fp16x2,fp16x1,fp32",
                    help="also time the step in these contraction modes (comma list; the headline's is "
                         "skipped; empty: none)")
    ap.add_argument("--p3", action="store_true",
                    help="time DS-GRFT with the acceleration rate (P = 3) on its 2.1e9-hypothesis grid (one JSON line)")
    ap.add_argument("--kt", action="store_true",
                    help="time the keystone branch (DS-KT-MFP map + detection) alone (one JSON line)")
    ap.add_argument("--kt-rows", type=int, default=0,
                    help="with --kt: the first N folding factors only (small profiling case)")
    ap.add_argument("--coarse-rm-steps", type=int, default=3,
                    help="timed calls of the standalone coarse-RM gather (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)
    if args.suite:
        return run_suite(args)
    if args.kt:
        return run_kt(args)
    if args.forms:
        return run_forms(args)
    if args.p3:
        print(json.dumps({"p3": measure_p3(args.steps, args.warmup, args.precision)}))
        return 0
    if args.pd:
        return run_pd(args)

    import torch
    import torch.distributed as dist

    import paper_2403_06788_gb300 as g
    import synth

    world, rank, local = rank_layout()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.load()

    sc = synth.ds_m512(run=rank)               # weak scaling: every rank owns its own CPI
    R, ds = sc.radar, sc.ds
    pg = ds.plain_equivalent()
    s = synth.make_echo(R, sc.targets, sc.seed)
    echo_host = torch.from_numpy(s).pin_memory()
    echo = echo_host.to(dev)
    ncell = ds.n_cells if args.cells <= 0 else min(args.cells, ds.n_cells)
    units = ds.r0_count * ncell * ds.n_fine * R.M
    nv, na = -(-ncell // ds.ac.count) * ds.Fv, ds.ac.count * ds.Fa    # v-slab holding the cells
    P = torch.empty((nv, na, ds.r0_count), dtype=torch.float32, device=dev)
    det_out = torch.zeros(args.topk * g._abi.DET_BYTES, dtype=torch.uint8, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    cfar = synth.CFAR(2, 16, 1e-6)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        g.dsgrft_fine_dfm(R, None, echo, ds, 0, ncell, args.precision, None, P)
        g.detect_peaks(P, cfar, args.topk, axes=pg, dr_m=R.dr_m, out=det_out, n_out=n_out)

    clk = ClockSampler(local).start()
    atexit.register(clk.stop)          # never leave nvidia-smi running
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = g.grft_sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

    # ---------------------------------------------------------------- timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    g.grft_timing(True)             # per-kernel CUDA events on the launching stream
    clk.begin()
    for i in range(args.steps):
        flush.fill_(i & 255)                                          # L2 flush, not timed
        e0, e1, e2 = ev[i]
        e0.record(stream)
        g.dsgrft_fine_dfm(R, None, echo, ds, 0, ncell, args.precision, None, P)
        e1.record(stream)
        g.detect_peaks(P, cfar, args.topk, axes=pg, dr_m=R.dr_m, out=det_out, n_out=n_out)
        e2.record(stream)
    torch.cuda.synchronize()
    clk.end()
    clk.stop()
    if world > 1:
        dist.barrier()
    ktime = {k: g.grft_timing_get(k) for k in ("tables", "split", "contract", "cfar", "topk")}
    g.grft_timing(False)
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    gemm_ms = [a.elapsed_time(b) for a, b, c in ev]
    det_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    st = g.grft_sync_status()
    dets, ndet = g.decode_detections(det_out, n_out, args.topk)
    # sampled (v, a) rows of the timed step's own power map (the P-only epilogue), every r0
    # bin, kept for the accuracy check against the oracle below (P is reused after this)
    rng = np.random.default_rng(1)
    vf = list(rng.integers(0, nv, ACC_ROWS)) + [int(round((t.v - pg.v.start) / pg.v.step)) for t in sc.targets]
    af = list(rng.integers(0, na, ACC_ROWS)) + [int(round((t.a - pg.a.start) / pg.a.step)) for t in sc.targets]
    vf, af = np.clip(vf, 0, nv - 1), np.clip(af, 0, na - 1)
    P_rows = P[torch.as_tensor(vf, device=dev), torch.as_tensor(af, device=dev)].cpu().numpy()

    # ---------------------------------------------------------------- end to end (host buffers)
    det_host = torch.empty_like(det_out, device="cpu").pin_memory()
    n_host = torch.empty(1, dtype=torch.int32).pin_memory()
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else max(3, args.steps // 2)
    e2e_tot = 0.0
    for i in range(e2e_steps):
        flush.fill_(i & 255)                 # L2 flushed as in the device-timed steps (not timed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        echo.copy_(echo_host, non_blocking=True)
        step()
        det_host.copy_(det_out, non_blocking=True)
        n_host.copy_(n_out, non_blocking=True)
        torch.cuda.synchronize()
        e2e_tot += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_tot / e2e_steps, dev)

    # ---------------------------------------------------------------- plain GRFT, same hypotheses
    plain_ms = plain_kernel_ms = plain_tables_ms = None
    # the plain grid restricted to the v-slab the DS step covers (the whole grid by default),
    # written into the same P buffer, whose shape it matches
    pg_slab = synth.PlainGrid(pg.r0_begin, pg.r0_count, synth.Axis(pg.v.start, pg.v.step, nv), pg.a)
    plain_units = nv * na * pg.r0_count * R.M
    assert tuple(P.shape) == (nv, na, pg.r0_count)
    if args.plain_steps > 0:
        g.grft_plain(R, echo, pg_slab, None, P)
        torch.cuda.synchronize()
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.grft_timing(True)                     # k_plain's own launches beside the whole call
        a_ev.record(stream)
        for _ in range(args.plain_steps):
            g.grft_plain(R, echo, pg_slab, None, P)
        b_ev.record(stream)
        torch.cuda.synchronize()
        plain_ms = a_ev.elapsed_time(b_ev) / args.plain_steps
        plain_kernel_ms = g.grft_timing_get("plain")[1] / args.plain_steps
        plain_tables_ms = g.grft_timing_get("tables")[1] / args.plain_steps
        g.grft_timing(False)
    # plain GRFT's error at this size: Y of the whole grid (the timed calls write P only)
    # against the oracle on sampled (v, a) rows, every r0 bin (targets' rows included)
    plain_err = None
    if args.plain_steps > 0 and rank == 0 and not args.no_cpu:
        import oracle
        rng = np.random.default_rng(2)
        pv = list(rng.integers(0, nv, ACC_ROWS // 4)) + [int(round((t.v - pg.v.start) / pg.v.step)) for t in sc.targets]
        pa = list(rng.integers(0, na, ACC_ROWS // 4)) + [int(round((t.a - pg.a.start) / pg.a.step)) for t in sc.targets]
        pv, pa = np.clip(pv, 0, nv - 1), np.clip(pa, 0, na - 1)
        Ypl = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device=dev)
        g.grft_plain(R, echo, pg_slab, Ypl, None)
        Yg = Ypl[torch.as_tensor(pv, device=dev), torch.as_tensor(pa, device=dev)].cpu().numpy()
        del Ypl
        torch.cuda.empty_cache()
        Ypo = oracle.grft_plain_rows(R, s, pg_slab, [int(x) for x in pv], [int(x) for x in pa])
        plain_err = float(np.abs(Yg - Ypo).max() / np.abs(Ypo).max())

    # ---------------------------------------------------------------- standalone coarse RM gather
    # (kernel a materialising Z = s[m][n0 + rho_c(m)] w_c(m) for every cell: HBM-write bound)
    crm_ms, crm_bytes = None, 0
    if args.coarse_rm_steps > 0:
        Z = torch.empty((ncell, R.M, ds.r0_count), dtype=torch.complex64, device=dev)
        g.dsgrft_coarse_rm(R, echo, ds, 0, ncell, Z)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.coarse_rm_steps):
            flush.fill_(1)
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record(stream)
            g.dsgrft_coarse_rm(R, echo, ds, 0, ncell, Z)
            b_ev.record(stream)
            torch.cuda.synchronize()
            tot += a_ev.elapsed_time(b_ev)
        crm_ms = tot / args.coarse_rm_steps
        crm_bytes = Z.numel() * 8 + echo.numel() * 8
        del Z
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- accuracy vs the oracle (sampled)
    acc = acc_p = None
    if rank == 0 and not args.no_cpu:
        import oracle
        from oracle.wrap import ds_rows_of_canonical
        cell, fine = ds_rows_of_canonical(ds, vf, af)
        Yo = oracle.dsgrft_rows(R, s, ds, cell, fine)
        Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device=dev)
        g.dsgrft_fine_dfm(R, None, echo, ds, 0, ncell, args.precision, Y, None)
        Yg = Y[torch.as_tensor(vf, device=dev), torch.as_tensor(af, device=dev)].cpu().numpy()
        del Y
        acc = float(np.abs(Yg - Yo).max() / np.abs(Yo).max())
        Po = np.abs(Yo) ** 2
        acc_p = float(np.abs(P_rows.astype(np.float64) - Po).max() / Po.max())

    # ---------------------------------------------------------------- the other contraction modes
    # (same step, same workload): bf16x3 / fp16x3 = hi/lo split of both operands, three
    # products per MAC; fp16x2 = hi/lo split of the gathered operand, the dechirp rounded once,
    # two products; fp16x1 = one FP16 product per MAC (not a split form); fp32 = the SIMT
    # contraction.  Each mode's value, contraction time, roofline and sampled error.
    others = {}
    modes = [m for m in str(args.other_precisions).split(",") if m and m != args.precision]
    if world == 1:
        for op in modes:
            def step_o():
                g.dsgrft_fine_dfm(R, None, echo, ds, 0, ncell, op, None, P)
                g.detect_peaks(P, cfar, args.topk, axes=pg, dr_m=R.dr_m, out=det_out, n_out=n_out)
            for _ in range(args.warmup if op != "fp32" else 1):
                step_o()
            torch.cuda.synchronize()
            k2 = max(3, args.steps // 2) if op != "fp32" else 3
            evo = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k2)]
            g.grft_timing(True)
            for i in range(k2):
                flush.fill_(i & 255)
                evo[i][0].record(stream)
                step_o()
                evo[i][1].record(stream)
            torch.cuda.synchronize()
            nco, mco = g.grft_timing_get("contract")
            g.grft_timing(False)
            ms_o = sum(a.elapsed_time(b) for a, b in evo) / k2
            err_o = None
            if rank == 0 and not args.no_cpu:
                Y = torch.empty((nv, na, ds.r0_count), dtype=torch.complex64, device=dev)
                g.dsgrft_fine_dfm(R, None, echo, ds, 0, ncell, op, Y, None)
                Yg = Y[torch.as_tensor(vf, device=dev), torch.as_tensor(af, device=dev)].cpu().numpy()
                del Y
                torch.cuda.empty_cache()
                err_o = float(np.abs(Yg - Yo).max() / np.abs(Yo).max())
            ent = {"products_per_mac": PRODUCTS_PER_MAC[op], "value": units / (1e-3 * ms_o),
                   "ms_per_step": ms_o, "max_rel_peak_err": err_o, "steps": k2}
            if nco > 0:                      # tensor-core modes: the contraction kernel's own events
                c_s = 1e-3 * mco / nco
                alg_o = FLOP_PER_HYP_PULSE * units / (nco / k2)
                peak_o = _peaks()[0].get("bf16_tflops", 1930.4)
                ent.update({"contract_ms": 1e3 * c_s, "roofline_frac": alg_o / c_s / 1e12 / peak_o,
                            "tensor_pipe_frac": alg_o * executed_per_algorithmic(op, ds.Fv, ds.Fa) / c_s / 1e12
                            / peak_o})
            others[op] = ent

    # ---------------------------------------------------------------- CPU oracle baseline
    cpu = None
    if rank == 0 and not args.no_cpu:
        v, cores, n, dt = _cpu_oracle_sample(sc, s, target_s=args.cpu_seconds)
        v1, _, n1, dt1 = _cpu_oracle_sample(sc, s, target_s=args.cpu_seconds / 3, warm_rows=2, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} (cell, fine) rows of the same DS grid x 4096 r0 x 512 pulses ({dt:.1f} s)",
               "value_1core": v1,
               "sample_1core": f"{n1} rows on one host thread ({dt1:.1f} s)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, src = _peaks()
    # the dominant kernel: the contraction (kernel b), timed by the library's per-kernel events
    # (the call runs it in rounds: per launch = the step's flops / launches per step)
    n_c, ms_c = ktime["contract"] if args.precision != "fp32" else (0, 0.0)
    if n_c > 0:
        gemm_avg_s = 1e-3 * ms_c / n_c
        launches_per_step = n_c / args.steps
    else:
        gemm_avg_s = 1e-3 * sum(gemm_ms) / len(gemm_ms)
        launches_per_step = 1
    alg_flops = FLOP_PER_HYP_PULSE * units / launches_per_step
    achieved = alg_flops / gemm_avg_s / 1e12
    exec_factor = executed_per_algorithmic(args.precision, ds.Fv, ds.Fa)   # executed / algorithmic FLOP
    # the timed region is a fraction of a second of back-to-back steps: the burst figure
    # (cuBLAS timed alone) is the denominator, not the seconds-long power-capped loop
    peak = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
    if args.precision == "fp32":
        # FP32 SIMT path: bound by FFMA issue, 152 SMs x 128 FMA/clk x 2 flop x max clock
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    value = job_rate(units, world, 1e-3 * total_ms / args.steps)
    # every hot kernel against its own bound: algorithmic bytes (HBM) or FLOP / event time
    hbm = peaks.get("hbm_gbs", 6678.5)
    fma_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    def _bw(name, nbytes, ms):
        if not ms:
            return None
        gbs = nbytes / (1e-3 * ms) / 1e9
        return {"bound": "hbm", "ms": ms, "achieved": gbs, "unit": "GB/s", "peak": hbm, "frac": gbs / hbm,
                "algorithmic_bytes": nbytes}
    hyps_step = nv * na * pg.r0_count
    kernel_rooflines = {
        "split (kernel a, split form)": _bw("split", ncell * ds.r0_count * R.M * 8 + echo.numel() * 8,
                                            ktime["split"][1] / args.steps if ktime["split"][0] else None),
        "cfar": _bw("cfar", hyps_step * 4, ktime["cfar"][1] / args.steps if ktime["cfar"][0] else None),
        "coarse_rm (kernel a, standalone)": _bw("coarse_rm", crm_bytes, crm_ms) if crm_ms else None,
        "plain_grft": None if plain_ms is None else {
            "bound": "fp32 fma", "kernel": "k_plain (CUDA events around its launches)", "ms": plain_kernel_ms,
            "achieved": 8 * plain_units / (1e-3 * plain_kernel_ms) / 1e12, "unit": "TFLOP/s", "peak": fma_peak,
            "frac": 8 * plain_units / (1e-3 * plain_kernel_ms) / 1e12 / fma_peak,
            "call_ms": plain_ms, "tables_ms": plain_tables_ms,
            "call_frac": 8 * plain_units / (1e-3 * plain_ms) / 1e12 / fma_peak},
    }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD if ncell == ds.n_cells else f"{WORKLOAD}, first {ncell} coarse cells",
                   "hypotheses": units // R.M, "pulses": R.M, "precision": args.precision,
                   "topk": args.topk, "cfar": "CA 2 guard / 16 train, pfa 1e-6",
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "parallelism": f"{world} independent CPI(s), one per GPU",
                   "range_migration": residual_migration(R, ds)},
        "roofline": {"bound": "tensor" if args.precision != "fp32" else "alu",
                     "kernel": ("k_ds_pair (tcgen05 split-operand contraction, pair form of mirrored fine "
                                "hypotheses, + |Y|^2 epilogue), CUDA events "
                                "around each launch on its stream" if n_c > 0 else
                                "dsgrft_fine_dfm call (tables + FP32 contraction)"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"{src} " + ("FP32 FFMA from SM count and max clock" if args.precision == "fp32"
                                                 else "bf16_tflops (burst)" + (" x 1 (dense FP16 and BF16 tensor "
                                                 "rates are equal)" if DTYPE[args.precision] == "f16" else "")),
                     "algorithmic_flop_per_launch": alg_flops, "executed_flop_per_launch": alg_flops * exec_factor,
                     "tensor_pipe_frac": alg_flops * exec_factor / gemm_avg_s / 1e12 / peak,
                     "traffic": (DRAM_TRAFFIC_PER_LAUNCH.get(args.precision)
                                 if (launches_per_step == 1 and args.cells == 0) else None),
                     "ms": 1e3 * gemm_avg_s,
                     "launches_per_step": launches_per_step},
        "stages_ms": dict({"dsgrft_fine_dfm call": sum(gemm_ms) / len(gemm_ms),
                           "detect_peaks call": sum(det_ms) / len(det_ms)},
                          **{f"{k} kernel": (v[1] / args.steps) for k, v in ktime.items() if v[0] > 0}),
        "plain_grft": None if plain_ms is None else {
            "value": plain_units / (1e-3 * plain_ms), "ms_per_step": plain_ms,
            "ds_speedup": (plain_ms / plain_units) / ((total_ms / args.steps) / units),
            "max_rel_peak_err": plain_err,
            "accuracy_sample": "%d (v, a) rows x %d r0 bins of the Y-writing call (random rows and the targets' rows)"
                               % (ACC_ROWS // 4 + len(sc.targets), pg.r0_count),
            "note": "both forms sum every pulse of every hypothesis (time-domain gather, no FFT): plain GRFT "
                    "executes 8 FP32 flop per hypothesis-pulse on the FMA pipes, the DS contraction "
                    "%.3g flop (products x 8 x slots per hypothesis of the pair form); the speedup is "
                    "the tensor cores and the pairing of mirrored hypotheses, not a shorter sum"
                    % (FLOP_PER_HYP_PULSE * exec_factor)},
        "kernels": kernel_rooflines,
        "max_rel_peak_err": acc,
        "max_rel_peak_err_power": acc_p,
        "accuracy_sample": None if acc is None else
            "%d (v, a) rows x %d r0 bins (%d random, the targets' rows): Y from the Y-writing call, "
            "P from the timed step's buffer against |Y|^2 of the oracle (relative to the peak power)"
            % (len(vf), ds.r0_count, ACC_ROWS),
        "other_precisions": others or None,
        "detections": {"total": ndet, "top1_p": float(dets["p"][0]) if len(dets) else None},
        "status": st,
        "e2e": {"value": job_rate(units, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": int(echo.numel() * 8),
                "d2h_bytes_per_step": int(det_out.numel() + 4)},
        "gpu_launches": sum(v[0] for v in ktime.values()),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
