#!/usr/bin/env python
"""Throughput of the fractional-step time step on one B300 (or N replicas).

Workload (default): 3-D decaying isotropic turbulence, periodic 128^3, random
solenoidal initial field with E(k) ~ k^4 exp(-2 (k/4)^2), u_rms = 1, nu = 1/400,
SSP-RK3 at CFL 0.5, mixed precision (FP32 stencils and transforms, FP64
tridiagonal / zero mode / reductions).  One "step" is one full time step
(three predictor + projection stages) through the C ABI.

Metric: cell-updates/s = cells x steps / time (higher is better).  L2 (126 MB)
is flushed before every timed step by writing a 256 MB buffer outside the
timed events; each step is timed with CUDA events on the solver's stream.

Also reported: the all-FP64 GPU path on the same workload with the relative L2
difference of the mixed result to it, the end-to-end number through host
buffers, the roofline of the dominant kernel, and the oracle timed on the
host cores (cpu_baseline).  --impl reference times the oracle alone.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

# Bytes each kernel must move per launch (every array read or written once), per cell
# of the 3-D mixed-precision step: FP32 fields and spectrum.  The predictor reads
# u (12) and writes u* (12), plus u^n (12) in RK3 stages 2 and 3; the y solve adds
# its FP64 tables (computed in roofline()).
def kernel_bytes_per_cell(name, dim, es, rk3):
    """Algorithmic bytes per cell of one launch: every array the kernel must touch read or written
    once (dim velocity fields and one scalar, es bytes per value).  The predictor of an RK3 step
    reads u^n as well in stages 2 and 3 (the average over the three stages); a transform pass or
    the spectral y solve reads and writes the scalar once.  The spectral y solve of 4096-row
    columns runs in three launches (fft_y_fwd, fft_y_solve, fft_y_inv): the solve's bytes are
    counted once, on fft_y_solve, and the two outer passes of its decomposition count none."""
    vb = es * dim
    if name in ("fft_y_fwd", "fft_y_inv"):
        return 0.0
    if name.startswith("predictor"):
        return (2 * vb + 3 * vb + 3 * vb) / 3.0 if rk3 else 2 * vb
    if name in ("fft_x_fwd_div", "fft_xz_fwd_div", "divergence"):
        return vb + es
    if name == "correct":
        return 2 * vb + es
    if name.startswith("fft_"):
        return 2.0 * es
    return None


# DRAM bytes (read + write) per launch from one ncu capture of the 128^3 mixed RK3
# workload (ncu flushes caches before each captured launch; writes still resident
# in L2 at kernel end are not counted; the predictor launch is an RK3 stage 2 or 3,
# which also reads u^n), keyed by kernel with the hash of the source files it was
# measured on (see KERNEL_SOURCES): a changed kernel reports traffic null until re-captured.
NCU_WORKLOAD = "isotropic_3d_128"   # the workload the traffic below was captured on
NCU_TRAFFIC = {
    "predictor": {"bytes": 50363136 + 1117952, "src": "787d2c94fc89"},
    "ysolve": {"bytes": 24119296 + 0, "src": "193f4010f1a6"},
    "fft_xz_fwd_div": {"bytes": 25194752 + 0, "src": "7e6f0662b6fd"},
    "fft_xz_inv": {"bytes": 8411904 + 0, "src": "7e6f0662b6fd"},
    "correct": {"bytes": 33560576 + 1024, "src": "96276b6b63ca"},
}


# The source a kernel's captured traffic was measured on: the text of the kernel
# (from a start marker to the end of its body) and the headers it builds on.
KERNEL_SOURCES = {
    "predictor": ("stencil.cu", "// Staged z-marching predictor", "if (!ok) atomicOr(status, 1u);", ["tma.cuh"]),
    "correct": ("stencil.cu", "__global__ void __launch_bounds__(kThreads) correct4_kernel", "\n}\n", []),
    "ysolve": ("poisson.cu", "// y solve for grids with many columns", "// Periodic y: the columns",
               ["fpconv.cuh", "tma.cuh"]),
    "fft_xz": ("fft_reg.cuh", "// x and z transforms of one y position j per block",
               "// The same fused x and z transforms with each y position's plane split", []),
    "fft": ("fft_reg.cuh", "", "", []),
}


def src_hash(name):
    for key, (fn, start, end, extra) in KERNEL_SOURCES.items():
        if name.startswith(key):
            csrc = os.path.join(ROOT, "paper_2505_23940_b300", "csrc")
            text = open(os.path.join(csrc, fn)).read()
            if start:
                i = text.index(start)
                text = text[i:text.index(end, i) + len(end)]
            m = hashlib.sha1(text.encode())
            for e in extra:
                m.update(open(os.path.join(csrc, e), "rb").read())
            return m.hexdigest()[:12]
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v, device):
    if ws == 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name):
    if name == "isotropic_3d_128":
        return S.isotropic_3d(n=128)
    if name == "isotropic_3d_256":
        return S.isotropic_3d(n=256)
    if name == "channel_3d":
        return S.channel_3d()
    if name == "taylor_green_2d":
        return S.taylor_green_2d()
    if name == "cylinder_2d":
        return S.cylinder_2d(seed=2, perturb=0.01)
    if name == "cylinder_array_2d":
        return S.cylinder_array_2d()
    if name.startswith("sweep_"):   # an HBM-sweep point ("sweep_384", "sweep_4096x4096")
        return sweep_workload(name[len("sweep_"):])[0]
    if name == "rough_channel_3d_128":
        # the rough-wall case of the static-box stress leg at 128^3 (cubes of 4 cells every 6, both
        # walls, markers every h/2)
        return S.rough_channel_3d(128, 128, 128, cube=4, pitch=6, both_walls=True, marker_spacing=0.5)
    raise ValueError(name)


def cpu_oracle_rate(wl, steps, threads=None):
    """Oracle (plain FP64 torch CPU) cell-updates/s over `steps` full steps of the workload."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O
    from helpers import body_of, grid_of, state_of
    if threads:
        torch.set_num_threads(threads)
    g = grid_of(wl)
    st = state_of(wl)
    body, params = body_of(wl)
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = O.step(g, st, wl.dt, scheme=wl.scheme, body=body, kernel=wl.kernel, params=params)
    dt = time.perf_counter() - t0
    return wl.cells() * steps / dt, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = workload(args.workload)
    threads = torch.get_num_threads()
    cpu_oracle_rate(wl, args.warmup)
    rate, secs = cpu_oracle_rate(wl, args.steps)
    line = {
        "impl": "reference", "metric": "cell-updates/s forward", "value": rate, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells": wl.cells(), "n": wl.n, "scheme": wl.scheme,
                   "precision": "FP64 throughout (the oracle)", "parallelism": "single"},
        "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
                         "sample": "%d full time steps of the %s workload (FP64 torch CPU oracle)"
                                   % (args.steps, args.workload)},
        "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_steps(g, u, dt, steps, flush, stream, body=None):
    times = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(u, dt, 1, body=body)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def kernel_times(g, u, dt, steps, flush, stream, filt, body=None):
    """Per-kernel CUDA-event times over `steps` flushed steps: every launch whose
    name starts with `filt` is bracketed by its own events on the grid's stream.
    Programmatic dependent launch is off for this pass, so that a launch's events
    enclose that launch alone (with it on, a kernel starts while its predecessor
    drains).  A separate pass from the timed region: events between launches
    would slow the step they measure."""
    g.set_tuning("pdl", 0)
    prof = None
    for _ in range(2):   # the first pass sizes the grid's event pool; the second is measured
        # a timed spin (about 50 ms) at the head of the stream: every instrumented launch is queued
        # before the GPU reaches it, so that no event interval contains host enqueue time
        torch.cuda._sleep(100_000_000)
        g.profile_begin(filt)
        timed_steps(g, u, dt, steps, flush, stream, body)
        prof = g.profile_end()
    g.set_tuning("pdl", 1)
    return prof


def ensemble_leg(args, flush):
    """Batched ensemble of 2-D cylinder flows of uneven size: K steps of every member through one
    CUDA-graph launch, against the same members launched one by one (mixed precision)."""
    import tempfile
    from paper_2505_23940_b300.ensemble import Ensemble
    os.environ.setdefault("FS_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "fsstep_tuning_bench.json"))
    wls = S.ensemble_cylinders(members=args.ensemble, seed=2, precision="mixed")
    ens = Ensemble(wls, "mixed", streams=32, tune=True)
    cells = ens.cells()
    k = args.steps
    snap = ens.snapshot()
    stream = torch.cuda.current_stream()
    ens.step_sequential(2)
    torch.cuda.synchronize()
    ens.restore(snap)
    flush.fill_(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step_sequential(k)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    ens.restore(snap)
    ens.capture(k)
    ens.restore(snap)
    ens.replay()   # the first replay uploads the graph: untimed, like any reused graph's
    ens.restore(snap)
    torch.cuda.synchronize()
    flush.fill_(4)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    ens.replay()
    e3.record(stream)
    torch.cuda.synchronize()
    g_ms = e2.elapsed_time(e3)
    sizes = sorted({tuple(w.n[:2]) for w in wls})
    # forward + adjoint over the workload's 500 steps (windows of 20: a checkpoint per window, each
    # window's forward recomputed in the reverse sweep); loss: the members' final kinetic energy
    window, windows = 20, 25
    weights = [[torch.tensor((w.xf[0][1] - w.xf[0][0]) ** 2, dtype=torch.float32, device="cuda")] * 2
               for w in wls]
    ens.restore(snap)
    ens.setup_adjoint(window, windows, weights)
    ens.capture_windows()
    ens.fwd_adj_graph()   # upload replays
    torch.cuda.synchronize()
    flush.fill_(5)
    e4, e5, e6 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e4.record(stream)
    ens.fwd_adj_graph()
    e5.record(stream)
    torch.cuda.synchronize()
    lam_graph = [[x.double().clone() for x in lu] for lu, _ in ens.lam_v]
    ens.fwd_adj_sequential()
    e6.record(stream)
    torch.cuda.synchronize()
    ga_ms, sa_ms = e4.elapsed_time(e5), e5.elapsed_time(e6)
    num = sum(float(((a - b.double()) ** 2).sum()) for la, (lu, _) in zip(lam_graph, ens.lam_v) for a, b in zip(la, lu))
    den = sum(float((b.double() ** 2).sum()) for lu, _ in ens.lam_v for b in lu)
    nfa = window * windows
    fwd_adj = {"steps": nfa, "window": window, "graph_launches": 2 * windows,
               "graph": {"value": cells * nfa / (ga_ms * 1e-3), "unit": "cell-updates/s fwd+adj", "ms": ga_ms},
               "one_by_one": {"value": cells * nfa / (sa_ms * 1e-3), "unit": "cell-updates/s fwd+adj", "ms": sa_ms},
               "speedup": sa_ms / ga_ms, "graph_vs_one_by_one_grad_rel_l2": (num / den) ** 0.5,
               "note": "every member's 500 steps forward (a checkpoint per 20-step window), then the reverse "
                       "sweep: per window its forward recomputed keeping each state and its 20 adjoint steps; "
                       "graph = 2 graphs over all members on 32 branches, 50 launches"}
    return {"members": len(wls), "cells": cells, "steps": k, "grid_sizes": len(sizes), "fwd_adj": fwd_adj,
            "graph": {"value": cells * k / (g_ms * 1e-3), "unit": "cell-updates/s", "ms": g_ms,
                      "launches": 1},
            "one_by_one": {"value": cells * k / (seq_ms * 1e-3), "unit": "cell-updates/s", "ms": seq_ms},
            "speedup": seq_ms / g_ms,
            "note": "every member advanced by K steps; graph = one CUDA-graph launch (after one untimed "
                    "upload replay) with members on 32 parallel branches; launch parameters autotuned per "
                    "grid size"}


def run_ours(args, ws, rank, local):
    from paper_2505_23940_b300 import grid_from_workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(args.workload)
    cells = wl.cells()
    stream = torch.cuda.current_stream()
    g = grid_from_workload(wl, args.precision, stream=stream)
    # "FP32 stencils / FP64 Poisson": on a periodic y the y part of the Poisson solve is the FP64
    # cyclic tridiagonal per x/z wavenumber (x and z transforms in FP32, zero mode exact)
    fp64_y = args.y_solve == "fp64" and wl.bc[1][0] == S.PERIODIC
    if fp64_y:
        g.set_tuning("y_spectral", 0)
    u0 = [torch.tensor(np.asarray(a), dtype=g.dtype, device=dev).contiguous() for a in wl.u0]
    u = [x.clone() for x in u0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if args.precision != "mixed":
        args.quick = True        # the comparison legs are defined for the mixed-precision headline
    from paper_2505_23940_b300 import body_tensor
    body = body_tensor(wl)   # FSI workloads (forward legs only)
    if body is not None:
        args.quick = True

    for _ in range(args.warmup):
        g.step(u, wl.dt, 1, body=body)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = g.launches()
    with Clocks(local) as clk:
        ms = timed_steps(g, u, wl.dt, args.steps, flush, stream, body=body)
    launches = g.launches() - launches0
    barrier(ws)
    total_ms = max_over_ranks(ws, sum(ms), dev)
    value = cells * args.steps * ws / (total_ms * 1e-3)

    # every kernel's launches timed by CUDA events on the grid's stream over the same K flushed
    # steps again: the dominant kernel and its roofline
    allk = kernel_times(g, u, wl.dt, args.steps, flush, stream, "", body=body)
    dominant = max(allk, key=lambda k: allk[k][1])
    cnt, kms = allk.get(dominant, (0, 0.0))
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6400.0)
    es = 4 if args.precision == "mixed" else 8
    bpc = kernel_bytes_per_cell(dominant, wl.dim, es, wl.scheme == "rk3")
    timing = ("CUDA events around every launch of the kernel over a second pass of the K timed "
              "steps (L2 flushed per step, programmatic dependent launch off in that pass)")

    def hbm_roofline(name):
        c, t = allk.get(name, (0, 0.0))
        b = kernel_bytes_per_cell(name, wl.dim, es, wl.scheme == "rk3")
        ach = b * cells / (t / c * 1e-3) / 1e9 if (c and b) else None
        tr = NCU_TRAFFIC.get(name) if args.workload == NCU_WORKLOAD else None
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak if ach else None,
                "traffic": tr["bytes"] if tr and tr.get("src") == src_hash(name) else None,
                "bytes_per_cell": b, "launches": c, "avg_launch_us": t / c * 1e3 if c else None,
                "timing": timing, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    if dominant == "ysolve":
        # the FP64 y solve is bound by the FP64 pipe.  Algorithmic FP64 flops per cell of the
        # cyclic twisted solve (periodic y): forward multiply-add 2, outward substitution 2 (FP32
        # fields: one multiply-add on the scaled rows, the scale applied in FP32 as the result is
        # narrowed; FP64 fields: multiply + multiply-add, 3), cyclic correction multiply-add 2 (an
        # upper bound: it is skipped where z is below FP64 rounding) = 6 (7); the wall-bounded
        # chain has no correction: 4 (5).  Peak: B300's nominal FP64 rate, 1.25 TFLOP/s (no FP64
        # peak is measured on this machine; a timing probe of independent DFMA chains reached
        # 1.06 TFLOP/s at 2032 MHz)
        flops = (2.0 if wl.bc[1][0] == S.PERIODIC else 0.0) + (4.0 if args.precision == "mixed" else 5.0)
        ach = flops * cells / (kms / cnt * 1e-3) / 1e12 if cnt else None
        tr = NCU_TRAFFIC.get(dominant) if args.workload == NCU_WORKLOAD else None
        roofline = {"kernel": dominant, "bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s",
                    "frac": ach / 1.25 if ach else None,
                    "traffic": tr["bytes"] if tr and tr.get("src") == src_hash(dominant) else None,
                    "flops_per_cell": flops,
                    "launches": cnt, "avg_launch_us": kms / cnt * 1e3 if cnt else None, "timing": timing,
                    "peak_source": "nominal FP64 rate (1.25 TFLOP/s); a DFMA timing probe reached 1.06"}
    else:
        roofline = hbm_roofline(dominant)
    stencil_roofline = hbm_roofline("predictor") if dominant != "predictor" else None

    line = {
        "metric": "cell-updates/s forward", "value": value, "unit": "cell-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "cells": cells, "n": wl.n, "scheme": wl.scheme,
                   "precision": ("FP64 throughout" if args.precision == "fp64" else
                                 "mixed: FP32 stencils and x/z transforms; FP64 Poisson along y (cyclic "
                                 "tridiagonal per wavenumber), zero mode and reductions" if fp64_y else
                                 "mixed (FP32 stencils/transforms, FP64 tridiagonal/zero mode/reductions)"),
                   "l2": "flushed before every timed step (256 MB write outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "gpu_launches": launches,
        "roofline": roofline,
        "stencil_roofline": stencil_roofline,
        "clocks": clk.summary(),
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in sorted(allk.items(), key=lambda kv: -kv[1][1])},
    }

    if not args.quick and fp64_y:
        # the same step with the y part of the Poisson solve as an FP32 DFT (zero mode exact)
        gs = grid_from_workload(wl, "mixed", stream=stream)
        us = [x.clone() for x in u0]
        for _ in range(args.warmup):
            gs.step(us, wl.dt, 1)
        mss = timed_steps(gs, us, wl.dt, args.steps, flush, stream)
        line["spectral_y"] = {"value": cells * args.steps / (sum(mss) * 1e-3), "unit": "cell-updates/s",
                              "ms_per_step": sum(mss) / args.steps,
                              "note": "the y part of the Poisson solve as an FP32 DFT with the exact zero mode "
                                      "(the same discrete solution; FP32 rounding in y)"}
        del gs, us

    if not args.quick:
        # all-FP64 GPU path on the same workload, and the mixed result's distance to it
        k64 = max(2, min(args.steps, 5))
        g64 = grid_from_workload(wl, "fp64", stream=stream)
        u64 = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev).contiguous() for a in wl.u0]
        for _ in range(2):
            g64.step(u64, wl.dt, 1)
        ms64 = timed_steps(g64, u64, wl.dt, k64, flush, stream)
        um = [x.clone() for x in u0]
        ud = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev).contiguous() for a in wl.u0]
        g.step(um, wl.dt, 10)
        g64.step(ud, wl.dt, 10)
        torch.cuda.synchronize()
        num = sum(float(((a.double() - b) ** 2).sum()) for a, b in zip(um, ud))
        den = sum(float((b ** 2).sum()) for b in ud)
        line["fp64_gpu"] = {"value": cells * k64 / (sum(ms64) * 1e-3), "unit": "cell-updates/s",
                            "ms_per_step": sum(ms64) / k64,
                            "mixed_vs_fp64_rel_l2_after_10_steps": (num / den) ** 0.5}
        line["speedup_mixed_over_fp64"] = line["value"] / ws / line["fp64_gpu"]["value"]
        del g64, u64

        # end to end through host buffers: H2D of the state from pinned memory, the step, D2H of the result
        host = [x.cpu().pin_memory() for x in u0]
        dev_u = [x.clone() for x in u0]
        nbytes = sum(x.numel() * x.element_size() for x in host)
        ev = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for d, h in zip(dev_u, host):
                d.copy_(h, non_blocking=True)
            g.step(dev_u, wl.dt, 1)
            for d, h in zip(dev_u, host):
                h.copy_(d, non_blocking=True)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        ems = max_over_ranks(ws, sum(a.elapsed_time(b) for a, b in ev), dev)
        line["e2e"] = {"value": cells * args.steps * ws / (ems * 1e-3), "unit": "cell-updates/s",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
        # forward + adjoint: K forward steps keeping snapshots, then the reverse sweep; the snapshot
        # count is chosen from free HBM (one per step here: no recomputation)
        from paper_2505_23940_b300.autodiff import Rollout
        ro = Rollout(g, wl.dt, args.steps)
        ua = [x.clone() for x in u0]
        # loss: final kinetic energy (1/2) sum u_T^2 h^3, whose adjoint is lam_T = u_T h^3
        vol = (2.0 * np.pi / wl.n[0]) ** 3
        lam_T = [x * vol for x in ro.forward(ua)[0]]
        ro.backward(ua, None, lam_T)        # warm-up of the adjoint kernels and buffers
        flush.fill_(7)
        torch.cuda.synchronize()
        ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        ea.record(stream)
        ro.forward(ua)
        eb.record(stream)
        ro.backward(ua, None, lam_T)
        ec.record(stream)
        torch.cuda.synchronize()
        fwd_ms, adj_ms = ea.elapsed_time(eb), eb.elapsed_time(ec)
        fa_ms = max_over_ranks(ws, fwd_ms + adj_ms, dev)
        slots = ro.used_slots
        line["fwd_adj"] = {"value": cells * args.steps * ws / (fa_ms * 1e-3), "unit": "cell-updates/s",
                           "steps": args.steps, "slots": slots, "recomputed_steps": ro.recomputed,
                           "recorded_stages": ro.recorded,
                           "forward_ms": fwd_ms, "reverse_ms": adj_ms,
                           "note": "K forward steps keeping snapshots (and, with recorded_stages, each "
                                   "step's RK3 stage states), then the reverse sweep (recomputation + adjoint "
                                   "steps)"}
        # the same with 4 snapshot slots: binomial recomputation in the reverse sweep
        ro4 = Rollout(g, wl.dt, args.steps, slots=4)
        lam4_T = [x * vol for x in ro4.forward(ua)[0]]
        torch.cuda.synchronize()
        ea.record(stream)
        ro4.forward(ua)
        ro4.backward(ua, None, lam4_T)
        eb.record(stream)
        torch.cuda.synchronize()
        r4_ms = max_over_ranks(ws, ea.elapsed_time(eb), dev)
        line["fwd_adj"]["revolve_4_slots"] = {"value": cells * args.steps * ws / (r4_ms * 1e-3),
                                              "unit": "cell-updates/s", "recomputed_steps": ro4.recomputed}
        del ro4, lam4_T
        # the same forward + adjoint on the all-FP64 path, and the distance of the mixed
        # gradient dJ/du_0 to it
        lam_mixed = ro.backward(ua, None, lam_T)[0]
        g64 = grid_from_workload(wl, "fp64", stream=stream)
        u64 = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev).contiguous() for a in wl.u0]
        ro64 = Rollout(g64, wl.dt, args.steps)   # the same snapshot policy as the mixed run
        lam64_T = [x * vol for x in ro64.forward(u64)[0]]
        torch.cuda.synchronize()
        ea.record(stream)
        ro64.forward(u64)
        lam64 = ro64.backward(u64, None, lam64_T)[0]
        eb.record(stream)
        torch.cuda.synchronize()
        f64_ms = max_over_ranks(ws, ea.elapsed_time(eb), dev)
        gnum = sum(float(((a.double() - b) ** 2).sum()) for a, b in zip(lam_mixed, lam64))
        gden = sum(float((b ** 2).sum()) for b in lam64)
        line["fwd_adj"]["fp64_gpu"] = {"value": cells * args.steps * ws / (f64_ms * 1e-3), "unit": "cell-updates/s",
                                       "ms": f64_ms,
                                       "mixed_vs_fp64_grad_rel_l2": (gnum / gden) ** 0.5}
        line["fwd_adj"]["speedup_mixed_over_fp64"] = line["fwd_adj"]["value"] / line["fwd_adj"]["fp64_gpu"]["value"]
        del g64, u64, ro64

    def leg(key, fn):
        # a leg that fails records its error instead of ending the run without the headline line
        try:
            line[key] = fn()
        except Exception as e:   # noqa: BLE001
            line[key] = {"error": "%s: %s" % (type(e).__name__, e)}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()

    if not args.quick and args.gradients:
        leg("gradients", lambda: gradient_legs(stream, flush))

    if not args.quick and args.ensemble > 0:
        leg("ensemble", lambda: ensemble_leg(args, flush))

    if not args.quick:
        leg("krylov", lambda: krylov_leg(wl, stream))
    if not args.quick and args.ib_stress:
        leg("ib_stress", lambda: ib_stress_leg(stream, flush))
        leg("ib2_stress", lambda: ib2_stress_leg(stream, flush))

    if not args.quick and args.sweep:
        leg("hbm_sweep", lambda: [sweep_leg(n, stream, flush) for n in args.sweep.split(",") if n])

    if rank == 0 and not args.quick and args.cpu_steps > 0:
        rate, secs = cpu_oracle_rate(wl, args.cpu_steps)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": torch.get_num_threads(),
                                "kind": "oracle",
                                "sample": "%d full time step(s) of the %s workload, FP64 torch CPU oracle, %.1f s"
                                          % (args.cpu_steps, args.workload, secs)}
    line["summary"] = summary_of(line)
    if rank == 0:
        print(json.dumps(line), flush=True)


def _face_weights(wl, dev, dtype):
    """Face control volumes per velocity component (x-fastest tensors): the weights of the
    kinetic energy 1/2 sum_c sum_faces u_c^2 V_c."""
    h = [np.diff(np.asarray(wl.xf[d], dtype=np.float64)) for d in range(wl.dim)]
    out = []
    for c in range(wl.dim):
        per = wl.bc[c][0] == S.PERIODIC
        ws = []
        for d in range(wl.dim):
            if d != c:
                ws.append(h[d])
            else:
                xc = 0.5 * (np.asarray(wl.xf[d][:-1]) + np.asarray(wl.xf[d][1:]))
                if per:
                    hf = np.empty_like(h[d])
                    hf[1:] = np.diff(xc)
                    hf[0] = xc[0] - (xc[-1] - (wl.xf[d][-1] - wl.xf[d][0]))
                else:
                    hf = np.empty(h[d].size + 1)
                    hf[1:-1] = np.diff(xc)
                    hf[0], hf[-1] = h[d][0], h[d][-1]
                ws.append(hf)
        w = ws[0][None, None, :] * ws[1][None, :, None]
        if wl.dim == 3:
            w = w * ws[2][:, None, None]
        out.append(torch.tensor(np.ascontiguousarray(w), dtype=dtype, device=dev))
    return out


def _fd_best(Jf, ad, steps):
    """Best relative agreement of central differences (J(+e) - J(-e)) / 2e with ad over steps e."""
    best, at = float("inf"), None
    for e in steps:
        fd = (Jf(e) - Jf(-e)) / (2.0 * e)
        r = abs(fd - ad) / max(abs(ad), 1e-300)
        if r < best:
            best, at = r, e
    return best, at


def gradient_legs(stream, flush):
    """The three gradient runs of the paper's workloads at full size (§2.4.1), forward + reverse
    through the revolve-checkpointed rollout, timed with CUDA events; each gradient checked along a
    seeded random direction against central differences of the FP64 GPU forward (best over a scan of
    steps), and the mixed gradient against the FP64 one.
      isotropic 128^3, SSP-RK3, 500 steps: J = final kinetic energy, dJ/du_0
      channel 192x129x128, forward Euler, 200 steps with 20 snapshot slots (revolve recomputation):
        J = final kinetic energy, dJ/df_x(y) (128 values)
      cylinder 640x320 FSI, 20000 steps: J = mean over the last 5000 steps of C_L^2, dJ/dk."""
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    from paper_2505_23940_b300.autodiff import Rollout
    dev = torch.device("cuda")
    out = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(stream)
        r = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return r, ev[0].elapsed_time(ev[1])

    # ---- isotropic turbulence 128^3, dJ/du_0 over 500 steps ----
    wl = S.isotropic_3d(n=128)
    n = 500
    cells = wl.cells()
    grads, res = {}, {}
    for prec in ("mixed", "fp64"):
        g = grid_from_workload(wl, prec, stream=stream)
        g.set_tuning("y_spectral", 0)
        dt_ = torch.float32 if prec == "mixed" else torch.float64
        u0 = [torch.tensor(np.asarray(a), dtype=dt_, device=dev).contiguous() for a in wl.u0]
        V = _face_weights(wl, dev, dt_)
        ro = Rollout(g, wl.dt, n)

        def run():
            uT = ro.forward(u0)[0]
            lam0, _ = ro.backward(u0, None, [x * v for x, v in zip(uT, V)])
            return lam0
        lam0, ms = timed(run)
        grads[prec] = [x.double() for x in lam0]
        res[prec] = {"ms": ms, "value": cells * n / (ms * 1e-3), "slots": ro.used_slots,
                     "recorded_stages": ro.recorded, "recomputed_steps": ro.recomputed}
        if prec == "fp64":
            V64 = V
            g64 = g
        else:
            del ro, g
        flush.fill_(1)
    rng = np.random.default_rng(11)
    d = [torch.tensor(rng.uniform(-1.0, 1.0, size=np.asarray(a).shape), device=dev) for a in wl.u0]
    u00 = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev) for a in wl.u0]

    def J_iso(e):
        u = [(a + e * b).contiguous() for a, b in zip(u00, d)]
        g64.step(u, wl.dt, n)
        return float(sum(0.5 * (x * x * v).sum() for x, v in zip(u, V64)))
    ad64 = float(sum((a * b).sum() for a, b in zip(grads["fp64"], d)))
    admx = float(sum((a * b).sum() for a, b in zip(grads["mixed"], d)))
    fd, at = _fd_best(J_iso, ad64, (1e-5, 1e-6, 1e-7, 1e-8))
    num = sum(float(((a - b) ** 2).sum()) for a, b in zip(grads["mixed"], grads["fp64"]))
    den = sum(float((b ** 2).sum()) for b in grads["fp64"])
    out["isotropic_128_500_steps"] = {
        "value": res["mixed"]["value"], "unit": "cell-updates/s fwd+adj", "ms": res["mixed"]["ms"],
        "fp64_value": res["fp64"]["value"], "mixed_slots": res["mixed"]["slots"],
        "recorded_stages": res["mixed"]["recorded_stages"], "recomputed_steps": res["mixed"]["recomputed_steps"],
        "fd_rel_err_fp64": fd, "fd_step": at,
        "fd_rel_err_mixed": abs(admx - ad64) / abs(ad64) if fd < 1e-4 else None,
        "mixed_vs_fp64_grad_rel_l2": (num / den) ** 0.5}
    del g64, grads, u00, d
    torch.cuda.empty_cache()

    # ---- channel 192x129x128, dJ/df_x(y) over 200 steps with 20 snapshot slots ----
    wl = S.channel_3d()
    n = 200
    cells = wl.cells()
    gf, res = {}, {}
    for prec in ("mixed", "fp64"):
        g = grid_from_workload(wl, prec, stream=stream)
        dt_ = torch.float32 if prec == "mixed" else torch.float64
        u0 = [torch.tensor(np.asarray(a), dtype=dt_, device=dev).contiguous() for a in wl.u0]
        V = _face_weights(wl, dev, dt_)
        ro = Rollout(g, wl.dt, n, slots=20)
        gfx = torch.zeros(wl.n[1], dtype=torch.float64, device=dev)

        def run():
            uT = ro.forward(u0)[0]
            ro.backward(u0, None, [x * v for x, v in zip(uT, V)], g_body_force=gfx)
            return gfx
        _, ms = timed(run)
        gf[prec] = gfx.clone()
        res[prec] = {"ms": ms, "value": cells * n / (ms * 1e-3), "recomputed_steps": ro.recomputed}
        if prec == "fp64":
            g64, V64 = g, V
        else:
            del ro, g
    dfx = torch.tensor(rng.uniform(-1.0, 1.0, size=wl.n[1]), device=dev)
    fx0 = torch.tensor(np.asarray(wl.body_force), device=dev)
    u00 = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev) for a in wl.u0]

    def J_ch(e):
        g64.set_body_force((fx0 + e * dfx).contiguous())
        u = [a.clone() for a in u00]
        g64.step(u, wl.dt, n)
        return float(sum(0.5 * (x * x * v).sum() for x, v in zip(u, V64)))
    ad64 = float((gf["fp64"] * dfx).sum())
    admx = float((gf["mixed"] * dfx).sum())
    fd, at = _fd_best(J_ch, ad64, (1e-2, 1e-3, 1e-4, 1e-5))
    out["channel_200_steps"] = {
        "value": res["mixed"]["value"], "unit": "cell-updates/s fwd+adj", "ms": res["mixed"]["ms"],
        "fp64_value": res["fp64"]["value"], "slots": 20, "recomputed_steps": res["mixed"]["recomputed_steps"],
        "fd_rel_err_fp64": fd, "fd_step": at, "fd_rel_err_mixed": abs(admx - ad64) / abs(ad64),
        "mixed_vs_fp64_grad_rel_l2": float((gf["mixed"] - gf["fp64"]).norm() / gf["fp64"].norm())}
    del g64, u00
    torch.cuda.empty_cache()

    # ---- cylinder FSI 640x320, dJ/dk over 20000 steps, J = mean of C_L^2 over the last 5000 ----
    wl = S.cylinder_2d(seed=2, perturb=0.01)
    n, m = 20000, 5000
    cells = wl.cells()
    k0 = float(wl.body.stiffness)
    gk, res, Jv = {}, {}, {}
    for prec in ("mixed", "fp64"):
        g = grid_from_workload(wl, prec, stream=stream)
        dt_ = torch.float32 if prec == "mixed" else torch.float64
        u0 = [torch.tensor(np.asarray(a), dtype=dt_, device=dev).contiguous() for a in wl.u0]
        b0 = body_tensor(wl)
        ro = Rollout(g, wl.dt, n)
        kk = torch.zeros(1, dtype=torch.float64, device=dev)

        def run():
            uT, bT, forces = ro.forward(u0, b0)
            lamF = torch.zeros_like(forces)
            lamF[n - m:, 1] = 8.0 * forces[n - m:, 1] / m        # J = (1/m) sum (2 F_y)^2
            ro.backward(u0, b0, [torch.zeros_like(x) for x in uT], torch.zeros_like(bT), lamF, g_stiffness=kk)
            return forces
        forces, ms = timed(run)
        Jv[prec] = float((4.0 * forces[n - m:, 1] ** 2).mean())
        gk[prec] = float(kk[0])
        res[prec] = {"ms": ms, "value": cells * n / (ms * 1e-3), "slots": ro.used_slots,
                     "recomputed_steps": ro.recomputed}
        if prec == "fp64":
            g64 = g
        else:
            del ro, g
        del forces

    # central differences over 20000 steps would see the epsilon mask flip at shifted steps (the
    # adjoint freezes it, A17); the FD pin runs the same FSI over 2000 steps, J over the last 1000
    nf, mf = 2000, 1000

    def J_cyl(e, want_grad=False):
        g64.set_stiffness(k0 + e)
        u = [torch.tensor(np.asarray(a), dtype=torch.float64, device=dev).contiguous() for a in wl.u0]
        ro = Rollout(g64, wl.dt, nf, slots=None if want_grad else 2)
        b0 = body_tensor(wl)
        _, bT, forces = ro.forward(u, b0)
        J = float((4.0 * forces[nf - mf:, 1] ** 2).mean())
        if not want_grad:
            return J
        kk = torch.zeros(1, dtype=torch.float64, device=dev)
        lamF = torch.zeros_like(forces)
        lamF[nf - mf:, 1] = 8.0 * forces[nf - mf:, 1] / mf
        ro.backward(u, b0, [torch.zeros_like(x) for x in u], torch.zeros_like(bT), lamF, g_stiffness=kk)
        return J, float(kk[0])
    _, gk_short = J_cyl(0.0, want_grad=True)
    fd, at = _fd_best(J_cyl, gk_short, (1e-4 * k0, 1e-5 * k0, 1e-6 * k0, 1e-7 * k0))
    g64.set_stiffness(k0)
    out["cylinder_fsi_20000_steps"] = {
        "value": res["mixed"]["value"], "unit": "cell-updates/s fwd+adj", "ms": res["mixed"]["ms"],
        "fp64_value": res["fp64"]["value"], "J": Jv["mixed"], "dJdk": gk["mixed"], "dJdk_fp64": gk["fp64"],
        "mixed_vs_fp64_dJdk_rel": abs(gk["mixed"] - gk["fp64"]) / abs(gk["fp64"]),
        "fd_rel_err_fp64": fd, "fd_step": at, "fd_horizon_steps": nf,
        "slots": res["mixed"]["slots"], "recomputed_steps": res["mixed"]["recomputed_steps"],
        "note": "FD pin (FP64 adjoint vs central differences of the FP64 forward) over 2000 steps, J over the "
                "last 1000; the 20000-step gradients are compared mixed vs FP64"}
    del g64
    torch.cuda.empty_cache()
    return out


def krylov_leg(wl, stream):
    """The paper's CG pressure solve (fs_solve_pressure_cg, FP64) against the direct solve on
    the workload's grid, for a seeded zero-mean right-hand side (compatible on periodic grids)."""
    from paper_2505_23940_b300 import grid_from_workload
    dev = torch.device("cuda")
    g = grid_from_workload(wl, "fp64", stream=stream)
    gen = torch.Generator(device="cpu").manual_seed(3)
    b = torch.rand(tuple(reversed(wl.n)), dtype=torch.float64, generator=gen).to(dev)
    b -= b.mean()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {}
    pd = g.solve_pressure(b)
    ev[0].record(stream)
    pd = g.solve_pressure(b)
    ev[1].record(stream)
    torch.cuda.synchronize()
    out["direct_ms"] = ev[0].elapsed_time(ev[1])
    for jac in (False, True):
        g.solve_pressure_cg(b, tol=1e-10, jacobi=jac, maxit=20000)
        ev[0].record(stream)
        p, it, rel = g.solve_pressure_cg(b, tol=1e-10, jacobi=jac, maxit=20000)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out["jacobi_cg" if jac else "cg"] = {
            "ms": ev[0].elapsed_time(ev[1]), "iterations": it, "relres": rel,
            "max_diff_to_direct_rel": float((p - pd).abs().max() / pd.abs().max())}
    out["note"] = "FP64 on the %s grid; tol 1e-10 on ||r|| / ||r0||" % wl.name
    del g
    return out


def support_faces(P, h, origin, ext, kind):
    """Number of distinct grid nodes of one face family (node k of direction d at origin[d] + k h[d],
    ext[d] nodes) in the union of the markers' delta-kernel supports (the nodes an IB kernel must
    read once): P (nm, d) marker positions."""
    width = 4 if kind == S.PESKIN4 else 3
    d = P.shape[1]
    first = []
    for a in range(d):
        sx = (P[:, a] - origin[a]) / h[a]
        first.append((np.floor(sx) - 1 if kind == S.PESKIN4 else np.floor(sx + 0.5) - 1).astype(np.int64))
    mask = np.zeros(int(np.prod(ext)), dtype=bool)
    offs = np.stack(np.meshgrid(*[np.arange(width)] * d, indexing="ij"), -1).reshape(-1, d)
    for o in offs:
        idx = [first[a] + o[a] for a in range(d)]
        ok = np.ones(P.shape[0], dtype=bool)
        for a in range(d):
            ok &= (idx[a] >= 0) & (idx[a] < ext[a])
        flat = np.zeros(int(ok.sum()), dtype=np.int64)
        stride = 1
        for a in range(d):
            flat += idx[a][ok] * stride
            stride *= ext[a]
        mask[flat] = True
    return int(mask.sum())


def ib2_stress_leg(stream, flush):
    """Moving 2-D immersed boundary at scale: a 12 x 116 array of cylinders (D = 24 cells, 75
    markers each: 104,400 markers, 1392 closed contours) moving as one elastically mounted body on a
    5760 x 624 grid, mixed precision, forward Euler.  Per IB kernel: time per launch and compulsory
    DRAM bytes (each array the kernel must touch, read or written once), hence achieved GB/s."""
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    dev = torch.device("cuda")
    wl = S.cylinder_array_2d()
    wl.body.w0 = (0.0, 0.01)
    nm = wl.body.X0.size
    nx, ny = wl.n[0], wl.n[1]
    h = wl.xf[0][1] - wl.xf[0][0]
    g = grid_from_workload(wl, "mixed", stream=stream)
    u = [torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous() for a in wl.u0]
    body = body_tensor(wl)
    for _ in range(2):
        g.step(u, wl.dt, 1, body=body)
    steps = 5
    ms = timed_steps(g, u, wl.dt, steps, flush, stream, body=body)
    prof = kernel_times(g, u, wl.dt, 2, flush, stream, "", body=body)
    peak = measured_peaks().get("hbm_gbs", 6400.0)
    # compulsory bytes per launch
    faces = (nx + 1) * ny + nx * (ny + 1)
    P = np.stack([wl.body.X0, wl.body.Y0 + wl.body.w0[1]], 1)
    x0 = wl.xf[0][0]
    sup = [support_faces(P, (h, h), (x0, x0 + 0.5 * h), (nx + 1, ny), wl.kernel),
           support_faces(P, (h, h), (x0 + 0.5 * h, x0), (nx, ny + 1), wl.kernel)]
    nib = int(g.ib_face_count())
    byt = {
        "classify_solid": faces * 1.0,                          # the flags written
        # flags read, IB bits and the list written; F_N: support flags, marker cell and fraction, wfac out
        "classify_ib_fn": faces * 1.0 + nib * (1.0 + 4.0) + sum(sup) * 1.0 + nm * (8.0 + 8.0 + 4.0 + 8.0),
        "ib_gather": nib * (4.0 + 8.0) + nm * (8.0 + 8.0 + 8.0),   # list, num/den out; marker cell, fraction, wfac
        "ib_force": sum(sup) * 4.0 + nm * (8.0 + 8.0 + 8.0 + 4.0 + 16.0),   # f on the supports; markers, q out
    }
    kern = {}
    for k, b in byt.items():
        if k not in prof:
            continue
        cnt, tot = prof[k]
        us = tot / cnt * 1e3
        kern[k] = {"us": us, "bytes": b, "GBs": b / (us * 1e-6) / 1e9, "frac": b / (us * 1e-6) / 1e9 / peak}
    out = {"n": [nx, ny], "cells": nx * ny, "markers": nm, "contours": len(wl.body.contours), "ib_faces": nib,
           "ms_per_step": sum(ms) / steps, "value": nx * ny * steps / (sum(ms) * 1e-3), "unit": "cell-updates/s",
           "markers_per_s_gather": nm / (kern["ib_gather"]["us"] * 1e-6) if "ib_gather" in kern else None,
           "ib_kernels": kern, "peak_GBs": peak,
           "kernels_ms_per_step": {k: v[1] / 2 for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
           "note": "compulsory bytes per launch: every array a kernel must touch, read or written once; the "
                   "support sets are the distinct faces within the markers' kernel supports"}
    del g, u
    torch.cuda.empty_cache()
    return out


def ib_stress_leg(stream, flush):
    """Static 3-D immersed boxes at scale: 256^3 rough-wall channel (cubes of 8 cells every 12 cells
    on both walls, markers every h/2: about 1.35 M markers), mixed precision, forward Euler."""
    from paper_2505_23940_b300 import grid_from_workload
    dev = torch.device("cuda")
    wl = S.rough_channel_3d(256, 256, 256, cube=8, pitch=12, both_walls=True, marker_spacing=0.5)
    nm = wl.boxes.X.shape[0]
    g = grid_from_workload(wl, "mixed", stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.set_boxes(wl.boxes.boxes, wl.boxes.X, wl.boxes.dV, wl.kernel)
    e1.record(stream)
    torch.cuda.synchronize()
    classify_ms = e0.elapsed_time(e1)
    u = [torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous() for a in wl.u0]
    del wl.u0
    for _ in range(2):
        g.step(u, wl.dt, 1)
    steps = 5
    ms = timed_steps(g, u, wl.dt, steps, flush, stream)
    prof = kernel_times(g, u, wl.dt, 2, flush, stream, "")
    cnt, tot = prof["ib3_force_gather"]
    gather_us = tot / cnt * 1e3
    # compulsory bytes of the gather: f (FP32) once on every face within some marker's kernel support
    # (neighbouring markers share most of them), the marker position and volume (32 B) and q (24 B)
    h = 2.0 / 256
    sup = 0
    for c in range(3):
        origin = [wl.xf[d][0] + (0.0 if d == c else 0.5 * h) for d in range(3)]
        ext = [256, 256, 256]
        if c == 1:
            ext[1] = 257
        sup += support_faces(wl.boxes.X, (h, h, h), origin, ext, wl.kernel)
    gbytes = sup * 4.0 + nm * (32 + 24)
    peak = measured_peaks().get("hbm_gbs", 6400.0)
    F = g.box_forces()
    out = {"n": [256, 256, 256], "cells": 256 ** 3, "markers": nm, "boxes": int(wl.boxes.boxes.shape[0]),
           "classify_ms": classify_ms, "ms_per_step": sum(ms) / steps,
           "value": 256 ** 3 * steps / (sum(ms) * 1e-3), "unit": "cell-updates/s",
           "force_gather_us": gather_us, "force_gather_markers_per_s": nm / (gather_us * 1e-6),
           "force_gather_bytes": gbytes, "support_faces": sup,
           "force_gather_GBs": gbytes / (gather_us * 1e-6) / 1e9,
           "force_gather_frac": gbytes / (gather_us * 1e-6) / 1e9 / peak,
           "kernels_ms_per_step": {k: v[1] / 2 for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
           "F": list(F)}
    del g, u
    torch.cuda.empty_cache()
    return out


def sweep_workload(spec):
    """The workload of one HBM-sweep point: spec "n": n^3 (the isotropic field up to 256^3, uniform
    random faces beyond, where the spectral generator costs minutes on the host); "AxB": a 2-D
    A x B periodic box with uniform random faces.  Returns (workload, [nx, ny, nz], field)."""
    if "x" in spec:
        nx, ny = (int(a) for a in spec.split("x"))
        wl = S.box_2d(nx, ny, (S.PERIODIC, S.PERIODIC), (S.PERIODIC, S.PERIODIC), Lx=2 * math.pi,
                      Ly=2 * math.pi * ny / nx, nu=1.0 / 400.0)
        dims, field = [nx, ny, 1], "uniform random faces"
    else:
        n = int(spec)
        if n <= 256:
            wl = S.isotropic_3d(n=n)
            field = "isotropic spectrum"
        else:
            wl = S.box_3d(n, n, n, (S.PERIODIC, S.PERIODIC), (S.PERIODIC, S.PERIODIC),
                          L=(2 * math.pi,) * 3, nu=1.0 / 400.0)
            field = "uniform random faces"
        dims = [n, n, n]
    if field != "isotropic spectrum":
        wl.u0 = S.random_fields(wl, 5, 1.0)
        wl.scheme = "rk3"
        wl.dt = 0.25 * 2 * math.pi / dims[0]
    return wl, dims, field


def sweep_leg(spec, stream, flush):
    """The RK3 step on a periodic grid whose working set exceeds L2 (`sweep_workload`): per-kernel
    times and the predictor's achieved HBM bandwidth."""
    from paper_2505_23940_b300 import grid_from_workload
    dev = torch.device("cuda")
    wl, dims, field = sweep_workload(spec)
    dim = wl.dim
    cells = dims[0] * dims[1] * dims[2]
    g = grid_from_workload(wl, "mixed", stream=stream)
    u = [torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous() for a in wl.u0]
    del wl.u0
    for _ in range(2):
        g.step(u, wl.dt, 1)
    steps = 5
    ms = timed_steps(g, u, wl.dt, steps, flush, stream)
    prof = kernel_times(g, u, wl.dt, 2, flush, stream, "")
    peak = measured_peaks().get("hbm_gbs", 6400.0)
    kms = {k: v[1] / 2 for k, v in prof.items()}
    cnt, tot = prof["predictor"]
    bpc = kernel_bytes_per_cell("predictor", dim, 4, True)
    ach = bpc * cells / (tot / cnt * 1e-3) / 1e9
    out = {"n": dims, "cells": cells, "field": field, "ms_per_step": sum(ms) / steps,
           "value": cells * steps / (sum(ms) * 1e-3), "unit": "cell-updates/s",
           "kernels_ms_per_step": dict(sorted(kms.items(), key=lambda kv: -kv[1])),
           "predictor": {"avg_launch_us": tot / cnt * 1e3, "bytes_per_cell": bpc, "achieved_GBs": ach,
                         "peak_GBs": peak, "frac": ach / peak}}
    # every kernel's algorithmic bytes per cell (FP32 fields, FP32 spectrum)
    step_bytes = sum((kernel_bytes_per_cell(k, dim, 4, True) or 0.0) * cells * prof[k][0] / 2 for k in kms)
    out["step_algorithmic_bytes"] = step_bytes
    out["step_GBs"] = step_bytes / (sum(ms) / steps * 1e-3) / 1e9
    out["step_frac"] = out["step_GBs"] / peak
    del g, u
    torch.cuda.empty_cache()
    return out


def summary_of(line):
    """The headline numbers of every leg in a few hundred bytes, printed last in the JSON line so
    that a truncated tail of the output still shows them."""
    def r(v, d=3):
        return None if v is None else float("%.*g" % (d, v))

    out = {"fwd": r(line.get("value")), "ms_step": r(line.get("ms_per_step")),
           ("ysolve_frac" if (line.get("roofline") or {}).get("kernel") == "ysolve" else "roofline_frac"):
               r((line.get("roofline") or {}).get("frac")),
           "stencil_frac": r((line.get("stencil_roofline") or {}).get("frac"))}
    if "spectral_y" in line:
        out["spectral_y"] = r(line["spectral_y"]["value"])
    if "fp64_gpu" in line:
        out["fp64"] = r(line["fp64_gpu"]["value"])
        out["mixed_vs_fp64_l2"] = r(line["fp64_gpu"]["mixed_vs_fp64_rel_l2_after_10_steps"], 2)
    if "e2e" in line:
        out["e2e"] = r(line["e2e"]["value"])
    if "fwd_adj" in line:
        fa = line["fwd_adj"]
        out["fwd_adj"] = r(fa["value"])
        out["fwd_adj_fp64"] = r(fa["fp64_gpu"]["value"])
        out["grad_mixed_vs_fp64"] = r(fa["fp64_gpu"]["mixed_vs_fp64_grad_rel_l2"], 2)
    line = {k: v for k, v in line.items() if not (isinstance(v, dict) and "error" in v)}
    for k, v in (line.get("gradients") or {}).items():
        out["grad_" + k] = {"v": r(v["value"]), "v64": r(v["fp64_value"]), "fd64": r(v["fd_rel_err_fp64"], 2),
                            "mx": r(v.get("fd_rel_err_mixed", v.get("mixed_vs_fp64_dJdk_rel")), 2)}
    if "ensemble" in line:
        e = line["ensemble"]
        out["ensemble"] = {"graph": r(e["graph"]["value"]), "one_by_one": r(e["one_by_one"]["value"]),
                           "speedup": r(e["speedup"]), "fa_graph": r(e["fwd_adj"]["graph"]["value"]),
                           "fa_one_by_one": r(e["fwd_adj"]["one_by_one"]["value"]),
                           "fa_speedup": r(e["fwd_adj"]["speedup"])}
    if "krylov" in line:
        out["cg_ms"] = r(line["krylov"]["cg"]["ms"])
    if "ib_stress" in line:
        out["ib3_gather_frac"] = r(line["ib_stress"].get("force_gather_frac"))
    if "ib2_stress" in line:
        out["ib2"] = {k: r(v["frac"]) for k, v in line["ib2_stress"]["ib_kernels"].items()}
        out["ib2_ms_step"] = r(line["ib2_stress"]["ms_per_step"])
    if "cpu_baseline" in line:
        out["cpu"] = r(line["cpu_baseline"]["value"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="isotropic_3d_128")
    ap.add_argument("--y-solve", default="fp64", choices=["fp64", "spectral"],
                    help="periodic y: FP64 cyclic tridiagonal (the FP64 Poisson of the 128^3 configuration) "
                         "or the FP32 DFT (also reported as the spectral_y leg)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the timed forward steps (fp64 implies --quick)")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--quick", action="store_true", help="timed forward steps only (for profiler runs)")
    ap.add_argument("--ensemble", type=int, default=64, help="members of the batched-ensemble leg (0: skip)")
    ap.add_argument("--sweep", default="256,384,512,4096x4096",
                    help="comma-separated out-of-L2 grids: n for n^3, AxB for a 2-D A x B box ('' to skip)")
    ap.add_argument("--ib-stress", type=int, default=1, help="run the 256^3 static-box leg (0: skip)")
    ap.add_argument("--gradients", type=int, default=1,
                    help="run the full-size gradient legs (isotropic 500 steps, channel 200, cylinder 20000; 0: skip)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
