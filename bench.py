#!/usr/bin/env python
"""Benchmark of the matrix-profile self-join on one GB300 (or N replicas).

Workload: self-join of a 2^20-sample float32 random walk with three planted
motif pairs and a planted discord, window m = 256, exclusion zone
ceil(m/2) = 128, in the FP32-mixed precision (FP64 statistics and distances;
FP32 diagonal recurrence and anchors on FP64-centred values).  One step = one whole mp_selfjoin
(input conversion, statistics, tile planning, the persistent diagonal-tile
kernel, finalize with the exact FP64 refine) on input already resident in
HBM.  The all-FP64 kernel is timed on the same input for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica of the workload (no collective on the data path); the timed region
is bracketed by a barrier and a synchronize, and the slowest rank's time is
reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "self-join Gcells/s @n=2^20,m=256: FP32-mixed vs FP64 GPU; % FP32 peak"
# --join lr: the same workload through the left/right-profile entry point
METRIC_LR = "left/right self-join Gcells/s @n=2^20,m=256 (FP32-mixed)"
METRIC_RAW = "non-normalised self-join Gcells/s @n=2^20,m=256 (FP32-mixed, tonal signal)"
METRIC_ANY = "anytime self-join, 5% run then resume to 100%, Gcells/s @n=2^20,m=256 (FP32-mixed)"
N_DEFAULT, M_DEFAULT, SEED = 1 << 20, 256, 2024
# DRAM traffic of one tile-kernel launch from an ncu capture, with the csrc digest it was taken at
PROFILE_TXT = os.path.join(ROOT, "profiles", "join_tile_f32_selfjoin_n2p20_m256.txt")
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def selfjoin_cells(l: int, E: int) -> int:
    """Admissible unordered pairs of a self-join: diagonals E..l-1."""
    k = l - E
    return k * (k + 1) // 2 if k > 0 else 0


# the sources the FP32 tile kernel is compiled from: a profile taken on other
# sources does not describe it
TILE_KERNEL_SOURCES = ("internal.cuh", "cand_f32.cuh", "join_tile.cuh", "join_fp32.cu")


def csrc_digest() -> str:
    """Digest of the tile kernel's code (comments and blank lines left out, so
    that editing a comment does not void a profile)."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1904_12626_gb300", "csrc")
    for f in TILE_KERNEL_SOURCES:
        with open(os.path.join(d, f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(f.encode() + code.encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        for line in (self.out or "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(REASONS, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, cells: int, steps: int, total_ms: float) -> float:
    """Whole-job Gcells/s: every rank joins its own copy of the workload (the
    self-join needs no exchange), timed by the slowest rank."""
    return world * cells * steps / (total_ms / 1e3) / 1e9


def workload(n: int, m: int):
    from paper_1904_12626_gb300 import synth
    x, info = synth.planted_walk(n, m, seed=SEED)
    return x, info


def cpu_oracle_rate(x, m: int, E: int, target_s: float, rows_min: int = 8):
    """Time the CPU oracle on a seeded sample of rows; returns
    (cells_per_s of the whole job extrapolated, rows, seconds, cores, results),
    results = (row indices, MP, PI, second-best distance) of the sample."""
    import numpy as np

    import oracle
    from paper_1904_12626_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    x64 = np.asarray(x, dtype=np.float64)
    l = len(x64) - m + 1
    cells = selfjoin_cells(l, E)
    rows = max(rows_min, cores)
    r0 = synth.sample_rows(l, rows, seed=99)
    t0 = time.perf_counter()
    res = [(r0, *oracle.selfjoin(x64, m, rows=r0))]
    dt = time.perf_counter() - t0
    if dt < target_s:
        more = int(rows * (target_s - dt) / max(dt, 1e-3))
        more = max(0, min(more, 64 * cores))
        if more:
            r1 = synth.sample_rows(l, more, seed=100)
            t1 = time.perf_counter()
            res.append((r1, *oracle.selfjoin(x64, m, rows=r1)))
            dt2 = time.perf_counter() - t1
            rows, dt = rows + more, dt + dt2
    per_row = dt / rows
    results = tuple(np.concatenate([r[k] for r in res]) for k in range(4))
    return cells / (per_row * l), rows, dt, cores, results


def accuracy(results, mp, pi, gap: float = 1e-3) -> dict:
    """Error of a GPU profile against the oracle on the oracle's rows: the
    largest |dMP|, and whether PI is identical on every row whose best and
    second-best distances differ by more than `gap`."""
    rows, mo, po, so = results
    g_mp, g_pi = np.asarray(mp)[rows], np.asarray(pi)[rows]
    fin = np.isfinite(mo)
    with np.errstate(invalid="ignore"):
        sep = fin & ((so - mo) > gap)
    return {"max_abs_dmp": float(np.max(np.abs(g_mp[fin] - mo[fin]))) if fin.any() else 0.0,
            "finite_pattern_equal": bool(np.array_equal(np.isfinite(g_mp), fin)),
            "separated_rows": int(sep.sum()),
            "pi_equal_on_separated": bool(np.array_equal(g_pi[sep], po[sep]))}


def stored_oracle_rows(x):
    """The oracle's answers on 4,096 seeded rows (plus every planted row +-4) of
    the planted 2^20 walk, as tests/golden/make_oracle_samples.py stored them
    (by running the oracle alone), when `x` is the input they were computed
    from (same fingerprint); else None."""
    path = os.path.join(ROOT, "tests", "golden", "c2_planted_n2p20_m256.npz")
    if not os.path.exists(path):
        return None
    a = np.ascontiguousarray(x)
    h = hashlib.sha256()
    h.update(str(a.dtype).encode() + str(a.shape).encode() + a.tobytes())
    z = np.load(path)
    if str(z["fingerprint"]) != h.hexdigest():
        return None
    return (z["rows"], z["mp"], z["pi"], z["sec"])


def merge_results(a, b):
    """Two (rows, mp, pi, sec) samples as one, each row once."""
    if b is None:
        return a
    rows = np.concatenate([a[0], b[0]])
    _, first = np.unique(rows, return_index=True)
    return tuple(np.concatenate([a[k], b[k]])[first] for k in range(4))


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_1904_12626_gb300 import synth  # noqa: F401 - input recipe only
    x, _ = workload(args.n, args.m)
    E = math.ceil(0.5 * args.m)
    l = args.n - args.m + 1
    cells = selfjoin_cells(l, E)
    for _ in range(args.warmup):
        cpu_oracle_rate(x, args.m, E, target_s=args.ref_step_s / 4)
    rates, rows_total, secs = [], 0, 0.0
    for _ in range(args.steps):
        r, rows, dt, cores, _ = cpu_oracle_rate(x, args.m, E, target_s=args.ref_step_s)
        rates.append(r)
        rows_total += rows
        secs += dt
    value = statistics.median(rates) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gcells/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": cells / (value * 1e9) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(args, E, cells),
        "cpu_baseline": {"value": value, "unit": "Gcells/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows_total} seeded rows of the n={args.n} self-join in "
                                   f"{secs:.1f} s, extrapolated to all {l} rows"},
        "e2e": {"value": value, "unit": "Gcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(args, E, cells):
    kind = {"lr": "left/right self-join", "anytime": "anytime self-join (5% run, resume to 100%)",
            "raw": "non-normalised self-join"}.get(getattr(args, "join", "self"), "self-join")
    data = "tonal signal (synth.tonal)" if getattr(args, "join", "self") == "raw" else "planted random walk"
    prec = "FP32-mixed" if args.prec == "fp32" else "FP64"
    return {"workload": f"{kind}, {data} n={args.n} float32, m={args.m}, ez=0.5 "
                        f"(E={E}), {prec}", "n": args.n, "m": args.m, "cells": cells,
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def workspace_tiles(ws) -> int:
    """Tiles the last join on workspace `ws` planned (the workspace header's
    tile count, bytes 24..31)."""
    return int(ws[24:32].cpu().numpy().view(np.uint64)[0])


def workspace_tile_diags(ws) -> int:
    """Diagonals per band of the tile shape the last join on `ws` ran (the
    workspace header's bytes 20..23): the library's choice when the variant
    was left to it."""
    return int(ws[20:24].cpu().numpy().view(np.int32)[0])


def fp64_roofline(cells, kernel_ms, anchor_fma, torch):
    """The all-FP64 tile kernel against the FP64 pipe, whose rate the library's
    probe measures on this GPU (mp_probe_fp64_rate: DFMA from independent
    chains).  Per cell 2 DFMA (the recurrence) + 1 DMUL (c invn_j), per row of
    8 cells one more DMUL (invn_i): 3.125 FP64 arithmetic ops; the anchors add
    m DFMA per diagonal per tile."""
    import ctypes

    from paper_1904_12626_gb300 import _lib
    rate = ctypes.c_double()
    _lib.check(_lib.load().mp_probe_fp64_rate(ctypes.byref(rate)), "mp_probe_fp64_rate")
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz") or 2070.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = rate.value / 1e12                                        # T FP64 lane-ops/s
    ops = 3.125 * cells + anchor_fma
    achieved = ops / (kernel_ms / 1e3) / 1e12
    return {"bound": "fp64", "achieved": achieved, "peak": peak,
            "unit": "T FP64 lane-ops/s (3.125 per cell: 2 DFMA, 1 + 1/8 DMUL; plus anchors)",
            "frac": achieved / peak, "anchor_dfma": anchor_fma,
            "anchor_share_of_ops": anchor_fma / ops,
            "peak_basis": (f"measured by mp_probe_fp64_rate on this GPU: "
                           f"{rate.value / (sms * f_max * 1e6):.2f} DFMA lanes/clk/SM at "
                           f"{f_max:.0f} MHz x {sms} SMs")}


def traffic_from_profile():
    """dram bytes (read + write) per tile-kernel launch, or None when the kernel
    sources changed since the capture."""
    if not os.path.exists(PROFILE_TXT):
        return None
    kv = {}
    with open(PROFILE_TXT) as fh:
        for line in fh:
            if ":" in line and not line.startswith((" ", "#", "|")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("csrc_sha") != csrc_digest():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_ours(args, world, rank, local):
    import torch

    from paper_1904_12626_gb300 import _lib, api, build
    build.build()
    api.init()
    lib = _lib.load()
    raw = args.join == "raw"
    if raw:                         # the non-normalised distance's domain: a bounded signal
        from paper_1904_12626_gb300 import synth
        x_np = synth.tonal(args.n, seed=SEED, dtype=np.float32)
    else:
        x_np, info = workload(args.n, args.m)
    n, m = args.n, args.m
    E = math.ceil(0.5 * m)
    l = n - m + 1
    cells = selfjoin_cells(l, E)
    x = torch.from_numpy(x_np).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    import ctypes
    tilekw = {"variant": args.variant, "tile_rows": args.tile_rows, "anchor_every": args.anchor_every}
    cfg = _lib.make_config(m, 0.5, args.prec, flags=_lib.MP_FLAG_RAW if raw else 0, **tilekw)
    lr = args.join == "lr"
    anytime = args.join == "anytime"
    need = (lib.mp_selfjoin_lr_workspace_bytes if lr else lib.mp_selfjoin_workspace_bytes)(
        n, ctypes.byref(cfg))
    ws = api.workspace(need, x.device)
    _lib.check(lib.mp_timing_enable(1), "mp_timing_enable")

    def join(xx, prec):
        """MP and PI (the left/right entry point returns both sides)."""
        if lr:
            return api.selfjoin_lr(xx, m, 0.5, prec, ws=ws)
        if anytime:                 # begin, a 5% run, then resume to the full profile
            run = api.Anytime(xx, m, seed=1, prec=prec, ws=ws)
            run.run(0.05)
            return run.run(1.0)
        return api.selfjoin(xx, m, 0.5, prec, raw=raw, ws=ws, **(tilekw if prec == args.prec else {}))

    def step(prec):
        return join(x, prec)

    for _ in range(args.warmup):
        step(args.prec)
    torch.cuda.synchronize()
    api.device_status(ws)

    # convert, descriptors, stats, fragile marking, key seeding (FP32: three kernels,
    # FP64: one), plan, tile kernel, fragile pass, finalize; anytime: begin (the same up
    # to the plan, plus the band order) and two runs (bind, window, tile kernel,
    # fragile pass, finalize)
    seed_launches = 3 if args.prec == "fp32" else 1
    launches_per_step = (7 + seed_launches + 10) if anytime else (8 + seed_launches)
    td = workspace_tile_diags(ws)                        # the shape the library ran
    kernel_name = (f"join_tile_kernel<Traits{args.prec.upper()}> "
                   f"{'variant ' + str(cfg.variant) if cfg.variant >= 0 else 'library choice'} "
                   f"({td} diagonals per band)")
    step_ms, kern_ms = [], []
    kms = ctypes.c_float()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            step(args.prec)
            e.record()
            e.synchronize()
            step_ms.append(s.elapsed_time(e))
            _lib.check(lib.mp_timing_last_ms(ctypes.byref(kms)), "timing")
            kern_ms.append(kms.value)
    torch.cuda.synchronize()
    barrier(world)
    api.device_status(ws)
    total_ms = max_over_ranks(sum(step_ms), world)
    kernel_ms = max_over_ranks(statistics.mean(kern_ms), world)
    tiles32 = workspace_tiles(ws)
    if anytime:                # the tile kernel runs twice per step: rate the whole step
        kernel_ms = total_ms / args.steps
    value = replica_value(world, cells, args.steps, total_ms)

    # all-FP64 kernel on the same input (comparison leg, one warm-up + timed steps)
    fp64 = None
    if not args.skip_fp64 and not lr and not anytime and not raw:
        cfg64 = _lib.make_config(m, 0.5, "fp64")
        ws64 = api.workspace(lib.mp_selfjoin_workspace_bytes(n, ctypes.byref(cfg64)), x.device)
        api.selfjoin(x, m, 0.5, "fp64", ws=ws64)
        torch.cuda.synchronize()
        t64 = []
        for _ in range(args.fp64_steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            api.selfjoin(x, m, 0.5, "fp64", ws=ws64)
            e.record()
            e.synchronize()
            t64.append(s.elapsed_time(e))
        _lib.check(lib.mp_timing_last_ms(ctypes.byref(kms)), "timing")
        ms64 = max_over_ranks(statistics.mean(t64), world)
        kern64 = kms.value
        fp64 = {"value": cells / (ms64 / 1e3) / 1e9, "unit": "Gcells/s", "ms_per_step": ms64,
                "kernel_ms": kern64}
        out64 = [t.cpu().numpy() for t in api.selfjoin(x, m, 0.5, "fp64", ws=ws64)]
        torch.cuda.synchronize()
        tiles64 = workspace_tiles(ws64)
        td64 = workspace_tile_diags(ws64)
        fp64["roofline"] = fp64_roofline(cells, kern64, tiles64 * td64 * m, torch)
        del ws64

    # end to end through the public API: pinned host input in, MP/PI back to host
    xh = torch.from_numpy(x_np).pin_memory()
    host_out = [torch.empty(l, dtype=dt).pin_memory()
                 for dt in ((torch.float64, torch.int64) * (2 if lr else 1))]
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        xd = xh.to("cuda", non_blocking=True)
        res = join(xd, args.prec)
        for k, (hbuf, dev) in enumerate(zip(host_out, res)):
            hbuf.copy_(dev, non_blocking=True)
        e.record()
        e.synchronize()
        if it >= args.warmup:
            e2e_ms.append(s.elapsed_time(e))
    e2e_total = max_over_ranks(sum(e2e_ms), world)
    e2e_value = world * cells * args.steps / (e2e_total / 1e3) / 1e9

    # the other join families at their parity-test sizes, library-default tiles
    # (batched and pan also as CUDA-graph replays), and the differentiable step
    families = None
    if args.families and not (lr or anytime or raw) and world == 1:
        families = {}
        peaks0 = measured_peaks()
        issue_peak0 = (torch.cuda.get_device_properties(0).multi_processor_count * 128 *
                       float(peaks0.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12)
        fsteps = max(3, min(args.steps, 3))
        with ClockSampler(local) as fclk:
            for fj in ("ab", "batched", "pan"):
                case = family_case(fj)
                res = time_family(case, {}, fsteps, 3, flush, graph=fj in ("batched", "pan"))
                families[fj] = family_summary(fj, case, res, {"tuned": False}, issue_peak0, world)
                del res
            families["grad"] = measure_grad(fsteps, 3, flush, issue_peak0)
        families["clocks"] = fclk.summary()
        families["steps"] = fsteps

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(0)
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz") or 2070.0)
    clocks = clk.summary()
    sms = props.multi_processor_count
    issue_peak = sms * 128 * f_max * 1e6 / 1e12            # T FP32 lane-instructions / s
    cells_per_s_kernel = cells / (kernel_ms / 1e3)
    achieved = 6 * cells_per_s_kernel / 1e12
    line = {
        "metric": (METRIC_LR if lr else METRIC_ANY if anytime else METRIC_RAW if raw else METRIC),
        "value": value, "unit": "Gcells/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 stats, centring and refine)",
        "data": "synthetic", "config": config_block(args, E, cells),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": issue_peak,
                     "unit": ("T FP32 lane-instructions/s (6 per cell: 2 FFMA, "
                              f"{'2 FADD' if raw else '2 FMUL'}, 2 FSETP)"),
                     "frac": achieved / issue_peak, "traffic": None if lr else traffic_from_profile(),
                     "kernel": kernel_name, "kernel_ms": kernel_ms,
                     "peak_basis": f"{sms} SMs x 128 lanes x {f_max:.0f} MHz "
                                   f"({'measured max clock' if peaks else 'nominal max clock'})",
                     "flop_frac": 6 * cells_per_s_kernel / (sms * 256 * f_max * 1e6),
                     "frac_at_median_clock": (achieved / (sms * 128 * clocks["sm_mhz"] * 1e6 / 1e12)
                                              if clocks.get("sm_mhz") else None),
                     "anchors": {"tiles": tiles32, "ffma": tiles32 * td * m,
                                 "ffma_per_cell": tiles32 * td * m / cells,
                                 "note": "dot products at each tile's first row: m FP32 "
                                         "multiply-adds per diagonal on values centred in "
                                         "FP64 (about 1.5 more FP32 instructions per term for "
                                         "the centring shift and the bound); their rounding "
                                         "widens the error bias"}},
        "fp64": fp64,
        "fp32_vs_fp64": (value / fp64["value"]) if fp64 else None,
        "e2e": {"value": e2e_value, "unit": "Gcells/s", "h2d_bytes_per_step": 4 * n,
                "d2h_bytes_per_step": 16 * l * (2 if lr else 1)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if families is not None:
        line["families"] = families
    if not args.skip_cpu and world == 1:
        rate, rows, secs, cores, results = cpu_oracle_rate(x_np, m, E, target_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate / 1e9, "unit": "Gcells/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{rows} seeded rows of the n={n} self-join in {secs:.1f} s, "
                                          f"extrapolated to all {l} rows"}
        if not (lr or anytime or raw):
            # error against the oracle on the rows it timed plus, for the planted
            # 2^20 walk, the 4,096-row sample it stored; FP32-mixed beside all-FP64
            stored = stored_oracle_rows(x_np) if (n, m) == (N_DEFAULT, M_DEFAULT) else None
            results = merge_results(results, stored)
            acc = {"rows": int(len(results[0])), "gap": 1e-3,
                   "tolerance": {"fp32_mixed": 1e-3, "fp64": 1e-9},
                   "sample": (f"{rows} rows timed now + {len(stored[0])} stored oracle rows "
                              "(tests/golden/c2_planted_n2p20_m256.npz)") if stored is not None
                             else f"{rows} rows timed now",
                   args.prec if args.prec == "fp64" else "fp32_mixed":
                       accuracy(results, host_out[0].numpy(), host_out[1].numpy())}
            if fp64 is not None:
                acc["fp64"] = accuracy(results, *out64)
            line["accuracy"] = acc
    print(json.dumps(line), flush=True)


def run_fluss(args, world, rank, local):
    """--join fluss: segmentation of the benchmark input's profile index (the
    self-join runs once, untimed); each step is one mp_fluss call with two
    boundaries, L2 flushed in between."""
    import ctypes

    import torch

    from paper_1904_12626_gb300 import _lib, api, build
    build.build()
    api.init()
    lib = _lib.load()
    x_np, _ = workload(args.n, args.m)
    m = args.m
    l = args.n - m + 1
    _, pi = api.selfjoin(torch.from_numpy(x_np).cuda(), m, 0.5, args.prec)
    ws = api.workspace(lib.mp_fluss_workspace_bytes(l), pi.device)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        api.fluss(pi, m, 2, ws=ws)
    api.device_status(ws)
    times = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            api.fluss(pi, m, 2, ws=ws)
            e.record()
            e.synchronize()
            times.append(s.elapsed_time(e))
    barrier(world)
    total_ms = max_over_ranks(sum(times), world)
    value = world * l * args.steps / (total_ms / 1e3) / 1e6
    # e2e: the profile index from pinned host memory, CAC and boundaries back
    pih = pi.cpu().pin_memory()
    cach = torch.empty(l, dtype=torch.float64).pin_memory()
    segh = torch.empty(2, dtype=torch.int64).pin_memory()
    e2e = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        pd = pih.to("cuda", non_blocking=True)
        c, g = api.fluss(pd, m, 2, ws=ws)
        cach.copy_(c, non_blocking=True)
        segh.copy_(g, non_blocking=True)
        e.record()
        e.synchronize()
        if it >= args.warmup:
            e2e.append(s.elapsed_time(e))
    e2e_total = max_over_ranks(sum(e2e), world)
    if rank != 0:
        return
    ms = total_ms / args.steps
    # algorithmic bytes per position: PI read 8, marks zeroed 4, two mark
    # atomics 8, marks read by both scan passes 8, CAC written 8, the
    # boundary search copies the curve (8 + 8) and reads it per boundary (2 x 8)
    bpp = 8 + 4 + 8 + 8 + 8 + 16 + 16
    achieved = bpp * l / (ms / 1e3) / 1e9
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    line = {
        "metric": "FLUSS positions/s @l=2^20 (corrected arc curve + 2 boundaries)",
        "value": value, "unit": "Mpositions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 counts, f64 curve", "data": "synthetic",
        "config": {"workload": f"FLUSS on the profile index of the planted random walk "
                               f"n={args.n}, m={m}", "l": l,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None,
                     "peak_basis": "measured copy bandwidth" if peaks else "fallback 6.8 TB/s"},
        "e2e": {"value": world * l * args.steps / (e2e_total / 1e3) / 1e6, "unit": "Mpositions/s",
                "h2d_bytes_per_step": 8 * l, "d2h_bytes_per_step": 8 * l + 16},
        "gpu_launches": 5 * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def measure_grad(steps, warmup, flush, issue_peak):
    """The differentiable step of the 2^16 walk (m = 128): FP32-mixed forward,
    loss = sum(MP) + mean of the 16 largest, backward scatter; eager steps,
    L2 flushed before each.  Returns the default run's summary object."""
    import ctypes

    import torch

    from paper_1904_12626_gb300 import _lib, api, synth
    lib = _lib.load()
    n, m = 1 << 16, 128
    cells = selfjoin_cells(n - m + 1, math.ceil(0.5 * m))
    x = torch.from_numpy(synth.random_walk(n, seed=58, dtype=np.float32)).cuda().requires_grad_(True)
    kms = ctypes.c_float()

    def step():
        x.grad = None
        prof, _ = api.matrix_profile(x, m)
        loss = prof.sum() + prof.topk(16).values.mean()
        loss.backward()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times, kern = [], []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        step()
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e))
        _lib.check(lib.mp_timing_last_ms(ctypes.byref(kms)), "timing")
        kern.append(kms.value)
    ms = statistics.mean(times)
    kernel_ms = statistics.mean(kern)
    return {"workload": f"random walk n={n} float32, m={m}, loss = sum(MP) + mean(top-16 MP), "
                        "forward + backward", "cells": cells, "ms_per_step": ms,
            "value": cells / (ms / 1e3) / 1e9, "unit": "Gcells/s", "kernel_ms": kernel_ms,
            "roofline_frac": 6 * cells / (kernel_ms / 1e3) / 1e12 / issue_peak}


def run_grad(args, world, rank, local):
    """--join grad: one differentiable step on a 2^16 random walk (float32,
    m = 128): the self-join forward (FP32-mixed), loss = sum(MP) + mean of
    the 16 largest MP values, and the backward kernel's scatter of the
    closed-form gradient through the argmin pairs.  The step is timed whole
    (forward, PyTorch's loss ops, backward); the tile kernel and the
    backward call are also timed alone."""
    import ctypes

    import torch

    from paper_1904_12626_gb300 import _lib, api, build, synth
    build.build()
    api.init()
    lib = _lib.load()
    _lib.check(lib.mp_timing_enable(1), "mp_timing_enable")
    n, m = 1 << 16, 128
    E = math.ceil(0.5 * m)
    l = n - m + 1
    cells = selfjoin_cells(l, E)
    x_np = synth.random_walk(n, seed=58, dtype=np.float32)
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    kms = ctypes.c_float()

    def step(xx):
        prof, _ = api.matrix_profile(xx, m)
        loss = prof.sum() + prof.topk(16).values.mean()
        loss.backward()
        return loss

    for _ in range(args.warmup):
        x.grad = None
        step(x)
    torch.cuda.synchronize()
    times, kern = [], []
    barrier(world)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            x.grad = None
            flush.fill_(1)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            step(x)
            e.record()
            e.synchronize()
            times.append(s.elapsed_time(e))
            _lib.check(lib.mp_timing_last_ms(ctypes.byref(kms)), "timing")
            kern.append(kms.value)
    barrier(world)
    total_ms = max_over_ranks(sum(times), world)
    kernel_ms = max_over_ranks(statistics.mean(kern), world)
    # the backward call alone (convert, window statistics, scatter kernel)
    with torch.no_grad():
        prof, pi = api.selfjoin(x.detach(), m)
        g = torch.ones_like(prof)
        g[torch.topk(prof, 16).indices] += 1.0 / 16
    bws = api.workspace(lib.mp_backward_workspace_bytes(n, m), x.device)
    bwd = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        api.backward(x.detach(), m, pi, g, ws=bws)
        e.record()
        e.synchronize()
        if it >= args.warmup:
            bwd.append(s.elapsed_time(e))
    api.device_status(bws)
    bwd_ms = max_over_ranks(statistics.mean(bwd), world)
    # end to end: pinned host series in, loss and gradient back to pinned host memory
    xh = torch.from_numpy(x_np).pin_memory()
    gh = torch.empty(n, dtype=torch.float32).pin_memory()
    lh = torch.empty((), dtype=torch.float32).pin_memory()
    e2e = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        xd = xh.to("cuda", non_blocking=True).requires_grad_(True)
        loss = step(xd)
        gh.copy_(xd.grad, non_blocking=True)
        lh.copy_(loss.detach(), non_blocking=True)
        e.record()
        e.synchronize()
        if it >= args.warmup:
            e2e.append(s.elapsed_time(e))
    e2e_total = max_over_ranks(sum(e2e), world)
    if rank != 0:
        return
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz") or 2070.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = sms * 128 * f_max * 1e6 / 1e12
    achieved = 6 * cells / (kernel_ms / 1e3) / 1e12
    line = {
        "metric": "differentiable self-join step (forward + backward) Gcells/s @n=2^16,m=128 "
                  "(FP32-mixed forward, FP64 backward)",
        "value": replica_value(world, cells, args.steps, total_ms), "unit": "Gcells/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 forward (FP64 stats, centring and refine), f64 backward",
        "data": "synthetic",
        "config": {"workload": f"random walk n={n} float32, m={m}, loss = sum(MP) + mean(top-16 MP)",
                   "cells": cells, "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": issue_peak,
                     "unit": "T FP32 lane-instructions/s (6 per cell: 2 FFMA, 2 FMUL, 2 FSETP)",
                     "frac": achieved / issue_peak, "traffic": None,
                     "kernel": "join_tile_kernel<TraitsFP32>, the library's tile shape (forward)",
                     "kernel_ms": kernel_ms},
        "backward": {"ms": bwd_ms, "rows": l, "fp64_atomic_adds": 2 * m * l,
                     "atomic_adds_per_s": 2 * m * l / (bwd_ms / 1e3)},
        "e2e": {"value": replica_value(world, cells, args.steps, e2e_total), "unit": "Gcells/s",
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n + 4},
        # forward: the eleven launches of an FP32-mixed join; backward: convert,
        # window statistics, scatter
        "gpu_launches": 14 * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def family_case(join: str, n_series: int = 4096):
    """Inputs and call of one join family at its parity-test size (AB: a 2^21
    walk against a 2^19 walk / white-noise mix with flat stretches, m = 512;
    batched: 4096 ragged walks of 1000..65536 samples, m in {32, 64, 128};
    pan: a 2^16 walk over 64 window sizes 16..1024).  Returns a dict with the
    host inputs, the admissible cells, a description, call(dev_inputs, kw) ->
    outputs, the output bytes, and the tuner entry point."""
    import torch

    from paper_1904_12626_gb300 import api, synth
    if join == "ab":
        m = 512
        a_np = synth.random_walk(1 << 21, seed=51, dtype=np.float32)
        b_np, _ = synth.mixed_with_flats(1 << 19, m, seed=52)
        la, lb = len(a_np) - m + 1, len(b_np) - m + 1
        return {"inputs": [a_np, b_np], "cells": la * lb, "out_bytes": 16 * (la + lb),
                "desc": f"AB-join, 2^21 random walk x 2^19 walk/white-noise mix with flat "
                        f"stretches, m={m}",
                "call": lambda xs, kw: api.abjoin(xs[0], xs[1], m, "fp32", **kw),
                "tune": lambda tuner, xs: tuner.abjoin(xs[0], xs[1], m)}
    if join == "batched":
        values, offsets, ms = synth.ragged_batch(n_series, seed=55)
        cells = 0
        for b in range(len(ms)):
            l_b = int(offsets[b + 1] - offsets[b]) - int(ms[b]) + 1
            cells += selfjoin_cells(l_b, math.ceil(0.5 * int(ms[b])))
        o_t = torch.from_numpy(offsets).cuda()
        m_t = torch.from_numpy(ms).cuda()
        max_m = int(ms.max())

        def call(xs, kw):
            mp, pi, _ = api.batched(xs[0], o_t, m_t, max_m=max_m, **kw)
            return mp, pi
        return {"inputs": [values], "cells": cells, "out_bytes": 16 * len(values),
                "desc": f"batched self-joins, {n_series} random walks of 1000..65536 samples, "
                        "m in {32,64,128}",
                "call": call,
                "tune": lambda tuner, xs: tuner.batched(xs[0], o_t, m_t, max_m=max_m)}
    n = 1 << 16
    ms = synth.pan_windows()
    x_np = synth.random_walk(n, seed=57, dtype=np.float32)
    cells = sum(selfjoin_cells(n - int(mk) + 1, math.ceil(0.5 * int(mk))) for mk in ms)
    return {"inputs": [x_np], "cells": cells, "out_bytes": 16 * len(ms) * (n - int(ms.min()) + 1),
            "desc": "pan profile, 2^16 random walk, 64 window sizes 16..1024",
            "call": lambda xs, kw: api.pan(xs[0], ms, **kw),
            "tune": lambda tuner, xs: tuner.pan(xs[0], ms)}


def time_family(case, kw, steps, warmup, flush, graph):
    """Eager steps (whole call, and the tile kernel alone), then, with `graph`,
    the same call recorded once in a CUDA graph and replayed per step; L2
    flushed before every timed step."""
    import ctypes

    import torch

    from paper_1904_12626_gb300 import _lib
    lib = _lib.load()
    dev_in = [torch.from_numpy(v).cuda() for v in case["inputs"]]
    call = case["call"]
    for _ in range(warmup):
        call(dev_in, kw)
    torch.cuda.synchronize()
    kms = ctypes.c_float()
    times, kern = [], []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        call(dev_in, kw)
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e))
        _lib.check(lib.mp_timing_last_ms(ctypes.byref(kms)), "timing")
        kern.append(kms.value)
    out = {"times": times, "kernel_ms": statistics.mean(kern), "dev_in": dev_in}
    if graph:
        _lib.check(lib.mp_timing_enable(0), "mp_timing_enable")   # no host events in a capture
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call(dev_in, kw)
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        gt = []
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            g.replay()
            e.record()
            e.synchronize()
            gt.append(s.elapsed_time(e))
        del g
        _lib.check(lib.mp_timing_enable(1), "mp_timing_enable")
        out["graph_times"] = gt
    return out


def family_summary(join, case, res, tile, issue_peak, world):
    """The per-family object of the bench line (eager and graph-replay times,
    the tile kernel against the issue roofline)."""
    ms = statistics.mean(res["times"])
    d = {"workload": case["desc"], "cells": case["cells"], "ms_per_step": ms,
         "value": case["cells"] / (ms / 1e3) / 1e9, "unit": "Gcells/s",
         "kernel_ms": res["kernel_ms"],
         "roofline_frac": 6 * case["cells"] / (res["kernel_ms"] / 1e3) / 1e12 / issue_peak,
         "tile": tile}
    if "graph_times" in res:
        gms = statistics.mean(res["graph_times"])
        d["graph_ms_per_step"] = gms
        d["graph_value"] = case["cells"] / (gms / 1e3) / 1e9
    return d


def run_family(args, world, rank, local):
    """--join ab | batched | pan: the other join families at their parity-test
    sizes, FP32-mixed, L2 flushed between steps, timed like the self-join
    (batched and pan also as CUDA-graph replays).  The autotuner first
    chooses the tile configuration on the same input (untimed; --no-tune keeps
    the library's defaults)."""
    import ctypes

    import torch

    from paper_1904_12626_gb300 import _lib, api, build
    build.build()
    api.init()
    lib = _lib.load()
    _lib.check(lib.mp_timing_enable(1), "mp_timing_enable")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    case = family_case(args.join, args.series)
    kw: dict = {}                   # tile configuration (the library's defaults with --no-tune)
    tile = {"tuned": False}
    if args.tune:                   # untimed: the autotuner chooses the tile configuration
        from paper_1904_12626_gb300.tune import Tuner
        tuner = Tuner(args.tune_cache or None, warmup=0, reps=1)   # the check run warms up
        kw.update(case["tune"](tuner, [torch.from_numpy(v).cuda() for v in case["inputs"]]))
        ch = tuner.last
        tile = {"tuned": True, **kw, "tuner_default_ms": ch.default_ms, "tuner_ms": ch.ms,
                "candidates_timed": ch.measured}
    barrier(world)
    with ClockSampler(local) as clk:
        res = time_family(case, kw, args.steps, args.warmup, flush,
                          graph=args.join in ("batched", "pan"))
    barrier(world)
    total_ms = max_over_ranks(sum(res["times"]), world)
    kernel_ms = max_over_ranks(res["kernel_ms"], world)
    host_in = [torch.from_numpy(v).pin_memory() for v in case["inputs"]]
    e2e = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        out = case["call"]([h.to("cuda", non_blocking=True) for h in host_in], kw)
        _ = [r.to("cpu", non_blocking=True) for r in out if r is not None]
        e.record()
        e.synchronize()
        if it >= args.warmup:
            e2e.append(s.elapsed_time(e))
    e2e_total = max_over_ranks(sum(e2e), world)
    if rank != 0:
        return
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz") or 2070.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = sms * 128 * f_max * 1e6 / 1e12
    cells = case["cells"]
    achieved = 6 * cells / (kernel_ms / 1e3) / 1e12
    fam = family_summary(args.join, case, res, tile, issue_peak, world)
    line = {
        "metric": f"{args.join} Gcells/s (FP32-mixed)",
        "value": replica_value(world, cells, args.steps, total_ms), "unit": "Gcells/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 stats, centring and refine)", "data": "synthetic",
        "config": {"workload": case["desc"], "cells": cells, "tile": tile,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": issue_peak,
                     "unit": "T FP32 lane-instructions/s (6 per cell: 2 FFMA, 2 FMUL, 2 FSETP)",
                     "frac": achieved / issue_peak, "traffic": None, "kernel_ms": kernel_ms},
        "e2e": {"value": replica_value(world, cells, args.steps, e2e_total), "unit": "Gcells/s",
                "h2d_bytes_per_step": int(sum(v.nbytes for v in case["inputs"])),
                "d2h_bytes_per_step": int(case["out_bytes"])},
        "gpu_launches": 11 * args.steps,
        "clocks": clk.summary(),
    }
    if "graph_ms_per_step" in fam:
        line["graph_ms_per_step"] = fam["graph_ms_per_step"]
        line["graph_value"] = fam["graph_value"]
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--join", choices=("self", "lr", "anytime", "raw", "fluss", "ab", "batched", "pan",
                                       "grad"),
                    default="self")
    # long aliases: under torchrun, --n / --m prefix-match the launcher's own options
    ap.add_argument("--n", "--series-length", dest="n", type=int, default=N_DEFAULT)
    ap.add_argument("--m", "--window", dest="m", type=int, default=M_DEFAULT)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=12.0)
    ap.add_argument("--variant", type=int, default=-1,
                    help="self-join tile variant (mp_variant_info; -1: the library's choice)")
    ap.add_argument("--tile-rows", type=int, default=0, help="self-join row-tile height (0: library's)")
    ap.add_argument("--anchor-every", type=int, default=0, help="self-join re-anchor interval (0: none)")
    ap.add_argument("--series", type=int, default=4096,
                    help="--join batched: number of series (a smaller batch for profiling)")
    ap.add_argument("--no-families", dest="families", action="store_false",
                    help="default run: skip the AB / batched / pan / gradient measurements")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="--join ab | batched | pan: keep the library's default tile configuration "
                         "(by default the autotuner chooses it first, untimed)")
    ap.add_argument("--tune-cache", default="",
                    help="JSON cache of the autotuner's choices (default: in memory only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if world > 1:
        args.gpus = world
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run = {"fluss": run_fluss, "ab": run_family, "batched": run_family,
               "pan": run_family, "grad": run_grad}.get(args.join, run_ours)
        run(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
