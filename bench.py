"""Benchmark: Voronoi cells/s on one (or N) GB300, FP32+FP64-recheck vs plain FP64.

One step = one whole tessellation (grid sort, kNN, clipping with every
re-queue pass, emit of neighbours + full geometry + volume + centroid) of the
1,048,576-point half-uniform / half-clustered cloud, inputs resident in HBM.

Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload mixed-1m|mixed-8m]
  python bench.py --impl reference ...   # the FP64 CPU oracle as the reference arm
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Voronoi cells/sec at 1M & 8M pts, 1 GB300: FP32+FP64-recheck vs plain FP64"
WORKLOADS = {
    "mixed-1m": dict(n=1 << 20, seed=1, desc="1,048,576 float32 points in [0,1)^3: 524,288 uniform + 524,288 in "
                     "1,000 isotropic Gaussian clumps (centres uniform, sigma log-uniform in [1e-3,1e-2], "
                     "out-of-box draws resampled), seed 1; k0=16 with doubling to k_max then the exhaustive pass; "
                     "outputs neighbours (CSR, original ids) + volume + centroid + full geometry"),
    "mixed-8m": dict(n=1 << 23, seed=2, sub_box=True, desc="8,388,608 float32 points, same recipe as mixed-1m, "
                     "seed 2; per-result errors of both forms against the FP64 oracle on the cells of a seeded "
                     "sub-box of about 65,536 generators"),
    "periodic-1m": dict(n=1 << 20, seed=5, periodic=True, desc="1,048,576 float32 points in the periodic unit box "
                        "[0,1)^3: the mixed-1m recipe (524,288 uniform + 524,288 in 1,000 Gaussian clumps) with "
                        "out-of-box draws wrapped by one period, so clumps continue across the faces, seed 5; cells "
                        "start as the cube of one period around their generator and are cut by the images of the "
                        "others; k0=16 with doubling to k_max then the exhaustive pass; outputs neighbours + volume "
                        "+ centroid + full geometry"),
    "mixed-300k": dict(n=300_000, seed=1, clumps=300, desc="300,000 float32 points, the mixed-1m recipe with 300 "
                       "clumps (a small case for profiler captures)"),
    "batch-512": dict(batch=True, seed=3, desc="512 independent point sets in [0,1)^3, sizes floor(10^U(3, log10 2e5)) "
                      "(about 18M points), each uniform or mixed-recipe clustered by a seeded coin flip, seed 3; "
                      "one CUDA graph per step (no-sync schedule), threads-per-cell / k0 / k_max / per-class grid "
                      "density autotuned on 64 seeded sets before the timed region; outputs neighbours + volume + "
                      "centroid"),
    "lloyd-1m": dict(lloyd=True, n=1 << 20, seed=4, desc="Lloyd relaxation of 1,048,576 uniform float32 points in "
                     "[0,1)^3 (seed 4); one step = one iteration: FP32-form tessellation with geometry, the moments "
                     "adjoint of sum_i M2_i (hand-written kernel through torch.autograd), and the update p <- p - "
                     "g / (2 V)"),
}
BATCH_SPACE = {"tpc": [16, 32], "k0": [12, 16, 24], "kmax_mult": [2], "rho": [1.0, 2.0, 3.0, 4.0, 6.0], "reps": 2}
# FP32 FMA peak from the unit counts and the maximum SM clock: 152 SMs x 128
# FP32 lanes x 2 flops x 2.070 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def _clip_traffic(n_cells: int):
    """DRAM bytes of the clip stage per step from a committed ncu capture,
    scaled to n_cells; None when the kernel source changed since the capture."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "clip_traffic.json")) as f:
            rec = json.load(f)
        src = open(os.path.join(ROOT, "paper_2412_04514_gb300", "csrc", "clip_impl.cuh"), "rb").read()
    except OSError:
        return None
    if hashlib.sha256(src).hexdigest() != rec.get("clip_impl_sha256"):
        return None
    return rec["bytes_per_cell"] * n_cells


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def dist_setup(gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def dist_max(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_oracle_rate(pts: np.ndarray, sample_cells: int, seed: int = 12345, sub_box: bool = False,
                    periodic: bool = False, one_core: bool = True) -> dict:
    """Times the FP64 CPU oracle on a sample of the workload's cells: random
    cells, or (sub_box) the cells of a seeded cube holding about that many
    generators. Returns the rate and the oracle's result for the sample."""
    import oracle

    if sub_box:
        from paper_2412_04514_gb300 import workloads as W

        idx = W.sub_box_cells(pts, sample_cells, seed)
        what = f"the {len(idx)} cells of a seeded sub-box"
    else:
        idx = np.sort(np.random.default_rng(seed).choice(len(pts), sample_cells, replace=False))
        what = f"{sample_cells} random cells"
    cores = oracle.default_threads()
    oracle.tessellate(pts[:2000], k0=16)  # load the library, warm the allocator
    t0 = time.perf_counter()
    r = oracle.tessellate(pts, k0=16, cells=idx, threads=cores, periodic=periodic)
    dt = time.perf_counter() - t0
    one_core_rate = None
    if one_core:  # the same oracle on one core, on the first tenth of the sample
        one = idx[: max(1, len(idx) // 10)]
        t1 = time.perf_counter()
        oracle.tessellate(pts, k0=16, cells=one, threads=1, periodic=periodic)
        dt1 = time.perf_counter() - t1
        one_core_rate = {"value": len(one) / dt1, "cells": int(len(one)), "seconds": dt1}
    return {"value": len(idx) / dt, "seconds": dt, "cores": cores, "flops_per_cell": float(oracle.clip_flops(r).mean()),
            "idx": idx, "result": r, "one_core": one_core_rate,
            "sample": f"{what} of the same {len(pts)}-point workload (kd-tree build included), FP64 oracle, "
                      f"{cores} threads"}


def errors_vs_oracle(cells, cpu: dict) -> dict:
    """Per-result error of a GPU tessellation on the oracle's sampled cells.

    Centroids: |dc| / |c| (the stated tolerance) and the stricter |dc| / V^(1/3).
    Neighbour lists that differ are classified: a difference made only of
    faces the oracle measures below 1e-6 V^(2/3) (or does not have) is a tiny
    face at a near-degenerate vertex; anything else is counted apart."""
    idx, w = cpu["idx"], cpu["result"]
    vol = cells.vol.cpu().numpy()[idx]
    cen = cells.cen.cpu().numpy()[idx]
    rv = np.abs(vol - w["vol"]) / w["vol"]
    dc = np.linalg.norm(cen - w["cen"], axis=1)
    rc = dc / np.linalg.norm(w["cen"], axis=1)
    sc = dc / np.cbrt(w["vol"])
    off, nbr = cells.nbr_off.cpu().numpy(), cells.nbr.cpu().numpy()
    tiny_only, other = 0, 0
    for a, i in enumerate(idx):
        g = nbr[off[i]:off[i + 1]]
        r = w["nbr"][w["nbr_off"][a]:w["nbr_off"][a + 1]]
        if np.array_equal(g, r):
            continue
        f0, f1 = w["face_off"][a], w["face_off"][a + 1]
        tags, areas = w["face_tag"][f0:f1], w["face_area"][f0:f1]
        lim = 1e-6 * w["vol"][a] ** (2 / 3)
        tiny = all((areas[tags == j].min() if np.any(tags == j) else 0.0) < lim
                   for j in set(g.tolist()) ^ set(r.tolist()))
        tiny_only += int(tiny)
        other += int(not tiny)
    return {"cells": int(len(idx)), "vol_rel_max": float(rv.max()), "vol_rel_median": float(np.median(rv)),
            "cen_rel_max": float(rc.max()), "cen_rel_median": float(np.median(rc)),
            "cen_over_size_max": float(sc.max()), "cen_over_size_median": float(np.median(sc)),
            "nbr_mismatch_cells": tiny_only + other, "nbr_mismatch_tiny_faces_only": tiny_only,
            "nbr_mismatch_other": other}


def run_reference(args, rank: int, world: int):
    """The reference arm: the FP64 CPU oracle on bounded samples, rank 0 only."""
    if rank != 0:
        return
    from paper_2412_04514_gb300 import workloads as W

    wl = WORKLOADS[args.workload]
    pts = W.mixed(wl["n"], wl["seed"], n_clumps=wl.get("clumps", 1000), periodic=wl.get("periodic", False))
    per_step = args.ref_cells
    for i in range(args.warmup):
        cpu_oracle_rate(pts, min(2000, per_step), seed=100 + i, periodic=wl.get("periodic", False), one_core=False)
    times = []
    cores = None
    for i in range(args.steps):
        # each step: the oracle's kd-tree over all points, then per_step random
        # cells, all host threads (the GPU arm's cpu_baseline times the same)
        r = cpu_oracle_rate(pts, per_step, seed=200 + i, periodic=wl.get("periodic", False), one_core=False)
        times.append(r["seconds"])
        cores = r["cores"]
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "n_points": wl["n"], "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random cells per step of the {wl['n']}-point workload (the "
                                   "oracle's kd-tree over all points built inside each step, as in the GPU arm's "
                                   "cpu_baseline), FP64 oracle, all host threads"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_tessellation(pts, params, steps: int, warmup: int, stage_times: bool, flush, world: int):
    """`steps` whole tessellations of the device points `pts` after `warmup`
    untimed ones, each timed with CUDA events on the launching stream, L2
    flushed before each. Returns (ms per step, stats per step, launches, the
    last step's cells)."""
    import torch

    import paper_2412_04514_gb300 as vt

    n = pts.shape[0]
    dev = pts.device
    ws = vt.Workspace(params, n, dev)
    p = vt.Params(**{**params.__dict__, "stage_times": stage_times})
    for _ in range(warmup):
        vt.tessellate(pts, p, workspace=ws)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    ms, stats = [], []
    launches0 = vt.launch_count()
    dist_barrier(world)
    torch.cuda.synchronize()
    cells = None
    for _ in range(steps):
        cells = None  # the previous step's outputs go back to the allocator first
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cells = vt.tessellate(pts, p, workspace=ws)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        stats.append(cells.stats)
    torch.cuda.synchronize()
    dist_barrier(world)
    launches = vt.launch_count() - launches0
    return ms, stats, launches, cells


def measure_8m(args, dev, flush, world: int, rank: int) -> dict:
    """The 8,388,608-point half of the metric: both forms on the mixed recipe
    (seed 2), FP32 steps, then FP64 steps, then (rank 0, one GPU) their errors
    against the oracle on a seeded sub-box of about 65,536 cells."""
    import torch

    import paper_2412_04514_gb300 as vt
    from paper_2412_04514_gb300 import workloads as W

    wl = WORKLOADS["mixed-8m"]
    n = wl["n"]
    pts_np = W.mixed(n, wl["seed"] + 1000 * rank, n_clumps=1000)
    pts = torch.from_numpy(pts_np).to(dev)
    emit = ("nbr", "vol", "cen", "geom")
    out = {"workload": wl["desc"]}
    keep = {}
    for prec in ("fp32", "fp64"):
        prm = vt.Params(precision=prec, k0=args.k0, k_max=args.k_max, threads_per_cell=32, emit=emit,
                        grid_density=args.rho)
        steps = args.steps_8m if prec == "fp32" else max(1, args.steps_8m - 1)
        ms, st, _, cells = time_tessellation(pts, prm, steps, 3, False, flush, world)
        tot = dist_max(sum(ms), world)
        out[prec] = {"value": n * world * len(ms) / (tot / 1e3), "unit": "cells/s", "ms_per_step": tot / len(ms),
                     "steps": len(ms), "warmup": 3, "status": st[-1]["status"]}
        keep[prec] = vt.Cells(vol=cells.vol, cen=cells.cen, nbr_off=cells.nbr_off, nbr=cells.nbr)
        cells = None
        torch.cuda.empty_cache()
    out["fp32_speedup"] = out["fp32"]["value"] / out["fp64"]["value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(pts_np, 65536, seed=17, sub_box=True)
        out["errors_vs_oracle"] = {"fp32_recheck": errors_vs_oracle(keep["fp32"], cpu),
                                   "fp64": errors_vs_oracle(keep["fp64"], cpu), "sample": cpu["sample"]}
    return out


def run_gpu(args, rank: int, world: int, local: int):
    import torch

    import paper_2412_04514_gb300 as vt
    from paper_2412_04514_gb300 import workloads as W

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    if wl.get("batch"):
        return run_batch(args, rank, world, local)
    if wl.get("lloyd"):
        return run_lloyd(args, rank, world, local)
    n = wl["n"]
    periodic = wl.get("periodic", False)
    pts_np = W.mixed(n, wl["seed"] + 1000 * rank, n_clumps=wl.get("clumps", 1000), periodic=periodic)
    pts = torch.from_numpy(pts_np).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    emit = ("nbr", "vol", "cen", "geom")

    def timed(params: vt.Params, steps: int, warmup: int, stage_times: bool):
        return time_tessellation(pts, params, steps, warmup, stage_times, flush, world)

    # warm up both forms, then time: FP32+recheck (headline) and plain FP64
    p32 = vt.Params(precision="fp32", k0=args.k0, k_max=args.k_max, threads_per_cell=32, emit=emit,
                    grid_density=args.rho, periodic=periodic)
    p64 = vt.Params(precision="fp64", k0=args.k0, k_max=args.k_max, threads_per_cell=32, emit=emit,
                    grid_density=args.rho, periodic=periodic)
    with Clocks(local) as clk:
        ms32, st32, launches32, cells = timed(p32, args.steps, args.warmup, stage_times=True)
    clocks = clk.summary()
    cells64 = None
    if args.steps_fp64 > 0:
        ms64, st64, _, cells64 = timed(p64, args.steps_fp64, 3, stage_times=True)
        tot64 = dist_max(sum(ms64), world)
        value64 = n * world * len(ms64) / (tot64 / 1e3)

    # the fused schedule (VT_FLAG_FUSED): kNN and clip in one walk, no lists
    cellsF = None
    if args.steps_fused > 0:
        pF = vt.Params(**{**p32.__dict__, "fused": True})
        msF, stF, _, cellsF = timed(pF, args.steps_fused, 3, stage_times=True)
        totF = dist_max(sum(msF), world)
        valueF = n * world * len(msF) / (totF / 1e3)
        wsF, ws32 = vt.workspace_size(pF, n), vt.workspace_size(p32, n)

    tot32 = dist_max(sum(ms32), world)
    value = n * world * len(ms32) / (tot32 / 1e3)

    # end to end through the public API with host buffers. Headline: a
    # pipelined stream (tessellate_stream) of clouds, every one copied in from
    # pinned host memory and its outputs copied back, the copies of one step
    # overlapping the tessellation of its neighbours. The stream runs over
    # warmup + steps + 1 clouds; the timed region is `steps` consecutive
    # results of its steady state (the pipeline filled by the warm-up results,
    # one more cloud behind the last timed one), each result's cloud copied in
    # and its outputs copied back. Beside it the serial figure of one
    # tessellate_host call after another
    host = torch.from_numpy(pts_np).pin_memory()
    e2e_stream_ms = None
    e2e_steps_ms = []
    if not args.no_e2e:
        stream = vt.tessellate_stream([host] * (args.warmup + args.steps + 1), p32, device=dev)
        for _ in range(args.warmup):
            out = next(stream)
            out = None
        dist_barrier(world)
        t0 = time.perf_counter()
        t_prev = t0
        for _ in range(args.steps):
            out = next(stream)
            out = None
            now = time.perf_counter()
            e2e_steps_ms.append(1e3 * (now - t_prev))
            t_prev = now
        e2e_stream_ms = dist_max(1e3 * (t_prev - t0), world)
        stream.close()
        torch.cuda.synchronize()
    e2e_ms = []
    h2d = host.numel() * 4
    d2h = 0
    out = None
    for i in range(args.warmup + args.steps if not args.no_e2e else 0):
        # a streaming caller hands each step's result on before the next call:
        # the pinned output buffers then return to torch's cache and are reused
        # (keeping the previous result alive makes a step pin 1.3 GB afresh)
        out = None
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = vt.tessellate_host(host, p32, device=dev)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        d2h = sum(getattr(out, f).numel() * getattr(out, f).element_size()
                  for f in ("vol", "cen", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                            "face_vtx") if getattr(out, f) is not None)
    e2e_tot = dist_max(sum(e2e_ms), world) if e2e_ms else 0.0
    e2e_value = n * world * len(e2e_ms) / (e2e_tot / 1e3) if e2e_ms else None
    out = None
    m8 = None
    if args.workload == "mixed-1m" and args.steps_8m > 0:
        with Clocks(local) as clk8:
            m8 = measure_8m(args, dev, flush, world, rank)
        m8["clocks"] = clk8.summary()

    if rank != 0:
        return

    # roofline of the dominant stage (the clipper), from the live event times
    stage = {k: statistics.mean(s[k] for s in st32) for k in ("ms_grid", "ms_knn", "ms_clip", "ms_emit")}
    peaks = _peaks()
    probe32, probe64 = vt.probe_fma("fp32"), vt.probe_fma("fp64")  # measured FMA rates (after the timed region)
    cpu = None
    errors = None
    if world == 1 and not args.no_cpu_baseline:
        sub = wl.get("sub_box", False)
        cpu = cpu_oracle_rate(pts_np, 65536 if sub else args.cpu_cells, seed=17 if sub else 12345, sub_box=sub,
                              periodic=periodic)
        errors = {"fp32_recheck": errors_vs_oracle(cells, cpu)}
        if cells64 is not None:
            errors["fp64"] = errors_vs_oracle(cells64, cpu)
        if cellsF is not None:
            errors["fused_fp32_recheck"] = errors_vs_oracle(cellsF, cpu)
        errors["sample"] = cpu["sample"]
    flops_per_cell = cpu["flops_per_cell"] if cpu else args.flops_per_cell
    clip_launches = statistics.mean(s["clip_launches"] for s in st32)
    achieved = n * flops_per_cell / (stage["ms_clip"] / 1e3) / 1e12
    roofline = {
        "kernel": "k_clip<float,32,2,64>%s (all passes of one step)" % (", periodic" if periodic else ""),
        "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None if periodic else _clip_traffic(n),
        "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (unit counts and max SM clock)",
        "peak_probe": {"fp32_tflops": probe32, "fp64_tflops": probe64,
                       "source": "vt_probe_fma: measured float32 / float64 FMA throughput of this GPU"},
        "units": f"{n} validated cells x {flops_per_cell:.0f} algorithmic FP32 flops/cell over {clip_launches:.1f} "
                 f"clip launches",
        "stage_ms": stage,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    # every stage against its own roofline (stage times of the timed FP32 steps)
    hbm = peaks.get("hbm_gbs") or 6764.0
    csr_bytes = sum(getattr(cells, f).numel() * getattr(cells, f).element_size()
                    for f in ("vol", "cen", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                              "face_vtx") if getattr(cells, f) is not None)
    kpre = 2 * args.k0 if 2 * args.k0 <= args.k_max else args.k0

    def hbm_line(nbytes, ms, what):
        gbs = nbytes / (ms / 1e3) / 1e9
        return {"bound": "hbm", "bytes": int(nbytes), "ms": ms, "achieved_gbs": gbs, "peak_gbs": hbm,
                "frac": gbs / hbm, "bytes_are": what}

    # the k-nearest-neighbour kernels against the FP32 peak: one squared
    # distance per candidate examined (3 subtractions, a product, two fused
    # multiply-adds: 8 flops), over their own CUDA-event time
    kl_ms = statistics.mean(s["ms_knn_lists"] for s in st32)
    cands = statistics.mean(s["knn_candidates"] for s in st32)
    queries = statistics.mean(s["knn_queries"] for s in st32)
    knn_tflops = cands * 8 / (kl_ms / 1e3) / 1e12 if kl_ms > 0 else None
    knn_alu = {"bound": "alu", "ms": kl_ms, "candidates_per_query": cands / max(queries, 1), "queries": int(queries),
               "flops_per_candidate": 8, "achieved_tflops": knn_tflops, "peak_tflops": FP32_PEAK_TFLOPS,
               "frac": None if knn_tflops is None else knn_tflops / FP32_PEAK_TFLOPS,
               "range_lists_ms": stage["ms_knn"] - kl_ms}
    stage_rooflines = {
        "grid_sort": hbm_line(52 * n, stage["ms_grid"], "52 B per point: points read twice, cell id and ticket "
                                                         "written and read, sorted float4 and permutation written"),
        "knn_and_range": hbm_line(n * (16 + 8 * kpre), stage["ms_knn"],
                                  f"the {kpre}-entry lists: 16 B query read + {kpre} x (4 B index + 4 B key) written "
                                  "(the stage also holds the range-list kernels, whose I/O is not counted; the "
                                  "stage is ALU- and latency-bound)"),
        "knn_alu": knn_alu,
        "clip": {"bound": "alu", "achieved_tflops": achieved, "peak_tflops": FP32_PEAK_TFLOPS,
                 "frac": achieved / FP32_PEAK_TFLOPS, "ms": stage["ms_clip"]},
        "emit": hbm_line(2 * csr_bytes + 16 * n, stage["ms_emit"],
                         "the per-cell records read (the outputs' bytes + a 16 B header) and the outputs written"),
    }
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": len(ms32),
        "warmup": args.warmup, "ms_per_step": tot32 / len(ms32), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "n_points": n, "precision": "fp32+fp64-recheck",
                   "k0": args.k0, "k_max": args.k_max, "grid_density": args.rho, "threads_per_cell": 32,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world} (independent clouds)"},
        "fp64_value": None if args.steps_fp64 <= 0 else value64,
        "fp32_speedup": None if args.steps_fp64 <= 0 else value / value64,
        "value_8m": None if m8 is None else m8["fp32"]["value"],
        "fp64_value_8m": None if m8 is None else m8["fp64"]["value"],
        "fp32_speedup_8m": None if m8 is None else m8["fp32_speedup"],
        "fused_value": None if cellsF is None else valueF,
        "fused_form": None if cellsF is None else {
            "value": valueF, "unit": "cells/s", "ms_per_step": totF / len(msF), "steps": len(msF),
            "schedule": "VT_FLAG_FUSED: every cell clips straight from its grid-shell walk (no neighbour lists)",
            "stage_ms": {k: statistics.mean(s[k] for s in stF) for k in ("ms_grid", "ms_knn", "ms_clip", "ms_emit")},
            "workspace_bytes_per_point": wsF / n, "list_schedule_workspace_bytes_per_point": ws32 / n},
        "fp64_form": None if args.steps_fp64 <= 0 else {
            "value": value64, "unit": "cells/s", "ms_per_step": tot64 / len(ms64), "steps": len(ms64),
            "stage_ms": {k: statistics.mean(s[k] for s in st64) for k in ("ms_grid", "ms_knn", "ms_clip", "ms_emit")},
            "fp32_speedup": value / value64},
        "e2e": None if not e2e_ms else {
            "value": n * world * args.steps / (e2e_stream_ms / 1e3), "unit": "cells/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": e2e_stream_ms / args.steps, "per_step_ms": e2e_steps_ms,
            "api": "steady state of a tessellate_stream over warmup + steps + 1 clouds: each timed result's cloud "
                   "copied in and its outputs copied out, overlapped with the neighbouring clouds' tessellation",
            "serial": {"value": e2e_value, "ms_per_step": e2e_tot / len(e2e_ms),
                       "api": "one tessellate_host call after another"}},
        "roofline": roofline,
        "stage_rooflines": stage_rooflines,
        "cpu_baseline": None if cpu is None else {"value": cpu["value"], "unit": "cells/s", "cores": cpu["cores"],
                                                  "kind": "oracle", "sample": cpu["sample"],
                                                  "one_core": cpu["one_core"]},
        "gpu_launches": int(launches32),
        "clocks": clocks,
        "errors_vs_oracle": errors,
        "passes": {"k_of_pass": st32[-1]["k_of_pass"], "cells_of_pass": st32[-1]["cells_of_pass"],
                   "clip_ms_of_pass": [statistics.mean(s["ms_clip_pass"][i] for s in st32)
                                       for i in range(len(st32[-1]["ms_clip_pass"]))],
                   "fp64_rechecks": st32[-1]["fp64_rechecks"], "precision_retries": st32[-1]["precision_retries"],
                   "capacity_retries": st32[-1]["capacity_retries"], "unvalidated": st32[-1]["unvalidated"]},
        "mixed_8m": m8,
    }
    print(json.dumps(line), flush=True)


def run_batch(args, rank: int, world: int, local: int):
    """The batch workload: the whole batch as one CUDA-graph replay per step."""
    import torch

    import paper_2412_04514_gb300 as vt
    from paper_2412_04514_gb300 import workloads as W

    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    pts_np, off, coin = W.batch_sets(seed=wl["seed"] + 1000 * rank)
    n = len(pts_np)
    pts = torch.from_numpy(pts_np).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    prm = vt.Params(precision="fp32", emit=("nbr", "vol", "cen"))
    t0 = time.perf_counter()
    b = vt.tuned_batch(pts, off, prm, space=BATCH_SPACE, sample_sets=64, seed=7)
    tune_s = time.perf_counter() - t0
    l0 = vt.launch_count()
    b.capture()
    per_replay = (vt.launch_count() - l0) // 2  # capture() runs once eagerly, then records
    for _ in range(args.warmup):
        b.replay()
    b.result()
    stream = torch.cuda.current_stream(dev)
    ms = []
    dist_barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.replay()
            e.record(stream)
            e.synchronize()
            ms.append(a.elapsed_time(e))
    clocks = clk.summary()
    torch.cuda.synchronize()
    dist_barrier(world)
    cells = b.result()
    tot = dist_max(sum(ms), world)
    value = n * world * len(ms) / (tot / 1e3)

    # end to end: pinned host points in, replay, results back to pinned host memory
    host = torch.from_numpy(pts_np).pin_memory()
    # pinned host buffers for every output (the neighbour array's length is
    # the batch's, the same every step)
    outs = {k: torch.empty(getattr(cells, k).shape, dtype=getattr(cells, k).dtype, pin_memory=True)
            for k in ("vol", "cen", "nbr_off", "nbr")}
    e2e_ms, d2h = [], 0
    for i in range(args.warmup + args.steps if not args.no_e2e else 0):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        b.points.copy_(host, non_blocking=True)
        b.replay()
        c = b.result()
        for k, v in outs.items():
            v.copy_(getattr(c, k), non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t1))
        d2h = sum(v.numel() * v.element_size() for v in outs.values())
    e2e_tot = dist_max(sum(e2e_ms), world) if e2e_ms else 0.0
    if rank != 0:
        return
    # stage split and roofline from one stage-timed run of the same tuned batch (synchronising schedule)
    sync = vt.tessellate_batch(pts, off, vt.Params(**{**b.params.__dict__, "no_sync": False, "stage_times": True}),
                               grid_res=b.grid_res).stats
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        big = int(np.argmax(np.diff(off)))
        sub = pts_np[off[big]:off[big + 1]]
        cpu = cpu_oracle_rate(sub, min(args.cpu_cells, len(sub)))
        cpu["sample"] += f" (set {big} of the batch, {len(sub)} points)"
    flops_per_cell = cpu["flops_per_cell"] if cpu else args.flops_per_cell
    achieved = n * flops_per_cell / (sync["ms_clip"] / 1e3) / 1e12
    tr = b.tune_report
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": len(ms),
        "warmup": args.warmup, "ms_per_step": tot / len(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "n_points": n, "n_sets": len(off) - 1, "precision": "fp32+fp64-recheck",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "tuned": {"threads_per_cell": b.params.threads_per_cell, "k0": b.params.k0,
                             "k_max": b.params.k_max, "density_of_class": tr["density_of_class"],
                             "class_counts": tr["class_counts"], "tune_seconds": tune_s,
                             "candidates": tr["n_tried"]}},
        "e2e": None if not e2e_ms else {
            "value": n * world * len(e2e_ms) / (e2e_tot / 1e3), "unit": "cells/s", "h2d_bytes_per_step": n * 12,
            "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_tot / len(e2e_ms)},
        "roofline": {
            "kernel": f"k_clip<float,{b.params.threads_per_cell},...> (all passes, stage-timed synchronising run)",
            "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (unit counts and max SM clock)",
            "stage_ms": {k: sync[k] for k in ("ms_grid", "ms_knn", "ms_clip", "ms_emit")}},
        "cpu_baseline": None if cpu is None else {"value": cpu["value"], "unit": "cells/s", "cores": cpu["cores"],
                                                  "kind": "oracle", "sample": cpu["sample"],
                                                  "one_core": cpu["one_core"]},
        "gpu_launches": int(per_replay * len(ms)),
        "clocks": clocks,
        "status": cells.stats["status"],
    }
    print(json.dumps(line), flush=True)


def run_lloyd(args, rank: int, world: int, local: int):
    """Lloyd iterations through the public API (vt.lloyd), one per step."""
    import torch

    import paper_2412_04514_gb300 as vt
    from paper_2412_04514_gb300 import workloads as W

    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    n = wl["n"]
    pts_np = W.uniform(n, wl["seed"] + 1000 * rank)
    p = torch.from_numpy(pts_np).to(dev)
    prm = vt.Params(precision="fp32")
    energies = []
    for _ in range(args.warmup):
        p = vt.lloyd(p, 1, prm, callback=lambda it, e: energies.append(e))
    stream = torch.cuda.current_stream(dev)
    ms = []
    l0 = vt.launch_count()
    dist_barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p = vt.lloyd(p, 1, prm, callback=lambda it, en: energies.append(en))
            e.record(stream)
            e.synchronize()
            ms.append(a.elapsed_time(e))
    clocks = clk.summary()
    launches = vt.launch_count() - l0
    torch.cuda.synchronize()
    dist_barrier(world)
    tot = dist_max(sum(ms), world)
    value = n * world * len(ms) / (tot / 1e3)
    # end to end: host points in, one iteration, new points and the loss back on the host
    host = torch.from_numpy(p.cpu().numpy()).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps if not args.no_e2e else 0):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d = host.to(dev, non_blocking=True)
        loss = []
        out = vt.lloyd(d, 1, prm, callback=lambda it, en: loss.append(en)).to("cpu")
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t1))
    e2e_tot = dist_max(sum(e2e_ms), world) if e2e_ms else 0.0
    if rank != 0:
        return
    # stage split of the forward tessellation of the current points (stage-timed)
    st = vt.tessellate(p, vt.Params(precision="fp32", emit=("vol", "cen", "m2", "geom"), stage_times=True)).stats
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(p.cpu().numpy(), args.cpu_cells)
    flops_per_cell = cpu["flops_per_cell"] if cpu else args.flops_per_cell
    achieved = n * flops_per_cell / (st["ms_clip"] / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": len(ms),
        "warmup": args.warmup, "ms_per_step": tot / len(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "n_points": n, "precision": "fp32+fp64-recheck",
                   "l2": "inputs larger than L2 (geometry of 1M cells, ~1 GB per step)",
                   "parallelism": f"replicas x{world}"},
        "lloyd": {"energy_first": energies[0], "energy_last": energies[-1], "iterations": len(energies),
                  "monotone": all(b <= a * (1 + 1e-9) for a, b in zip(energies, energies[1:]))},
        "e2e": None if not e2e_ms else {
            "value": n * world * len(e2e_ms) / (e2e_tot / 1e3), "unit": "cells/s", "h2d_bytes_per_step": n * 12,
            "d2h_bytes_per_step": n * 12 + 8, "ms_per_step": e2e_tot / len(e2e_ms)},
        "roofline": {
            "kernel": "k_clip<float,32,2,64> of the forward tessellation (stage-timed run)",
            "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (unit counts and max SM clock)",
            "stage_ms": {k: st[k] for k in ("ms_grid", "ms_knn", "ms_clip", "ms_emit")}},
        "cpu_baseline": None if cpu is None else {"value": cpu["value"], "unit": "cells/s", "cores": cpu["cores"],
                                                  "kind": "oracle", "sample": cpu["sample"] + " (tessellation only)",
                                                  "one_core": cpu["one_core"]},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--steps-fp64", type=int, default=3)
    ap.add_argument("--steps-fused", type=int, default=5, help="steps of the fused schedule (0: skip)")
    ap.add_argument("--steps-8m", type=int, default=3, help="steps of the 8M half of the metric (0: skip)")
    ap.add_argument("--workload", default="mixed-1m", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-cells", type=int, default=100_000)
    ap.add_argument("--ref-cells", type=int, default=100_000)
    ap.add_argument("--flops-per-cell", type=float, default=25134.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--k0", type=int, default=16)
    ap.add_argument("--k-max", type=int, default=32)
    ap.add_argument("--rho", type=float, default=2.0)
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
