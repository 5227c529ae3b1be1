#!/usr/bin/env python
"""Benchmark of the P2M++ query path on GB300.

One step = one closest-point query pass (nearest site + interception-list scan, every
query answered) over the workload's full query set, inputs resident in HBM.  Default
workload: icosphere(6) with 3-octave value noise (81,920 triangles), 10M queries (half
uniform in the 1.2x bbox, half surface + N(0, (0.01 diag)^2)).  The index is built once
before timing; its CSR build time is reported separately, as are fwd+bwd throughput on the
differentiation workload (icosphere(5), 1M near-surface queries, L = sum d^2) and the
end-to-end rate through the host-buffer C-ABI call.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --impl reference the FP64 brute-force oracle is timed
on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import p2m_workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM = 128
# algorithmic FP32 work model (FLOP, an FMA counts 2): a candidate site is a squared
# distance and a compare, a list entry the bounding-sphere test, an exact test the weighted
# mix of the interior and edge paths of the point-triangle distance, and a query its fixed
# grid lookup, bound setup and result
FLOP_PER_SITE = 8
FLOP_PER_ROW_ENTRY = 10
FLOP_PER_EXACT = 80
FLOP_PER_QUERY = 26
BYTES_PER_QUERY = 12 + 32  # FP32 point in; dist, closest[3], tri, bary[3] out

WORKLOADS = {
    "large": ("icosphere(6) + 3-octave noise a=0.05, 81,920 tris; 10M queries: 50% uniform in 1.2x bbox, "
              "50% surface + N(0,(0.01 diag)^2); seed 0", lambda n: W.workload_large(n or 10_000_000)),
    "small": ("UV sphere 32x16, 960 tris; 100k queries uniform in 1.2x bbox; seed 0",
              lambda n: W.workload_small(n or 100_000)),
    "symmetric": ("cylinder+cone 512x128, 203,776 tris, aux on; 10M queries: 70% within 0.02 diag of the surface, "
                  "30% uniform in 1.2x bbox; seed 0", lambda n: W.workload_symmetric(n or 10_000_000)),
    "diff": ("icosphere(5) + noise, 20,480 tris; 1M queries surface + N(0,(0.01 diag)^2); seed 0",
             lambda n: W.workload_diff(n or 1_000_000)),
}


def reduce_max_ms(ms, world, device=None):
    """Step time of the slowest rank (every rank calls this; world == 1 returns ms)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(n_per_rank, ms, world):
    """Whole-job queries/s of `world` replicas that each answer n_per_rank queries per step."""
    return world * n_per_rank / (ms / 1e3)


def metric_name(config):
    return "closest-point queries/s (10M pts, 82k tris)" if config == "large" else f"closest-point queries/s ({config})"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.15)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Kernels of this library launched by one query pass (CUB's scan / select / sort kernels and
# memsets not counted).  Sorted schedules 0 and 4: k_cell_rank, k_cell_scatter, the scan
# kernel(s) (k_query_thread, or k_query_sites + k_query_scan), k_query_warp, k_split_records,
# k_bvh_closest.  Schedules 1-3 (unsorted): k_query_thread, k_query_warp, k_bvh_closest.
# Schedule 5 (site-staged): k_site_rank, k_site_scatter, k_query_staged, k_query_warp,
# k_split_records, k_bvh_closest.
OWN_KERNELS_PER_STEP = {0: 6, 1: 3, 2: 3, 3: 3, 4: 7, 5: 6}


def query_source_hash():
    """First 16 hex digits of the SHA-256 of the query-kernel sources (query.cu,
    query_dev.cuh, geom.cuh) with comments and blank lines removed: the code the profiled
    kernels were compiled from."""
    import hashlib
    import re

    def strip(src):
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    srcs = [os.path.join(ROOT, "paper_2605_00429_gb300", "csrc", f) for f in ("query.cu", "query_dev.cuh", "geom.cuh")]
    return hashlib.sha256("\n".join(strip(open(f).read()) for f in srcs).encode()).hexdigest()[:16]


def profile_fields(config):
    """The machine-readable fields ("- key: value" lines) of the committed ncu summary of this
    workload, if it was taken on the current query-kernel code (else an empty dict)."""
    path = os.path.join(ROOT, "profiles", f"k_query_{config}.md")
    try:
        h = query_source_hash()
        fields = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip()
    except OSError:
        return {}
    return fields if fields.get("source_sha256_16") == h else {}


def profiled_traffic(config, n):
    """DRAM bytes per query pass from the committed ncu summary, scaled to n queries (None if
    the summary is not of the current sources)."""
    try:
        return float(profile_fields(config)["dram_bytes_per_query"]) * n
    except (KeyError, ValueError):
        return None


def profiled_l1tex_pct(config):
    """L1TEX throughput of k_query_thread (% of peak) in the same summary, or None."""
    try:
        return float(profile_fields(config)["l1tex_throughput_pct"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(mesh, q, target_s=12.0, seed=0):
    """The FP64 oracle (as it stands) on a bounded random sample of the workload's queries."""
    import oracle
    rng = np.random.default_rng(seed + 99)
    probe = q[rng.choice(len(q), min(len(q), 256), replace=False)]
    t = time.perf_counter()
    oracle.closest(mesh.verts, mesh.tris, probe)
    per_q = max((time.perf_counter() - t) / len(probe), 1e-9)
    n = int(min(len(q), max(256, target_s / per_q)))
    sample = q[rng.choice(len(q), n, replace=False)]
    t = time.perf_counter()
    oracle.closest(mesh.verts, mesh.tris, sample)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} random queries of the workload, FP64 brute force over all {mesh.n_tris} triangles",
            "seconds": dt}


def config_leg(p2m, key, dev, steps, schedule, flush, hbm_peak):
    """One more workload of the contract, measured like the headline: build time, then the
    query pass timed with CUDA events over `steps` steps (L2 flushed between steps)."""
    import torch
    desc, make = WORKLOADS[key]
    mesh, q = make(0)
    n = q.shape[0]
    t0 = time.perf_counter()
    idx = p2m.P2MIndex(mesh.verts, mesh.tris, schedule=schedule)
    build_ms = (time.perf_counter() - t0) * 1e3
    st = idx.stats()
    pts = torch.from_numpy(q).to(dev)
    out = (torch.empty(n, device=dev), torch.empty(n, 3, device=dev), torch.empty(n, device=dev, dtype=torch.int32),
           torch.empty(n, 3, device=dev))
    for _ in range(3):
        idx.query(pts, out=out)
    cnt = idx.counters(pts)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        idx.query(pts, out=out)
        b.record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    del idx
    return {"workload": desc, "queries": n, "tris": mesh.n_tris, "queries_per_s": n / (ms / 1e3), "ms_per_step": ms,
            "steps": steps, "build_wall_ms": build_ms, "csr_build_ms": st["ms_tri"] + st["ms_lbvh"] + st["ms_k1"],
            "grid_build_ms": st["ms_grid"], "sites": st["n_sites"], "aux_sites": st["n_aux_sites"],
            "avg_list": st["avg_row"], "max_list": st["max_row"],
            "queried_list": cnt["queried_list"] / n,
            "queried_entries": cnt["row_entries"] / n, "queried_exact": cnt["exact_tests"] / n,
            "hbm_frac": BYTES_PER_QUERY * n / (ms / 1e3) / 1e9 / hbm_peak}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle timed on the host cores, same metric."""
    if rank != 0:
        return
    desc, make = WORKLOADS[args.config]
    mesh, q = make(args.queries)
    import oracle
    oracle.build()
    steps, warm = args.steps, args.warmup
    rng = np.random.default_rng(5)
    probe = q[rng.choice(len(q), 256, replace=False)]
    t = time.perf_counter()
    oracle.closest(mesh.verts, mesh.tris, probe)
    per_q = (time.perf_counter() - t) / 256
    budget = 150.0 / max(1, steps + warm)  # the whole run stays within a few minutes
    n = int(max(64, min(len(q), budget / max(per_q, 1e-9))))
    times = []
    for k in range(warm + steps):
        sample = q[rng.choice(len(q), n, replace=False)]
        t = time.perf_counter()
        oracle.closest(mesh.verts, mesh.tris, sample)
        if k >= warm:
            times.append(time.perf_counter() - t)
    ms = float(np.mean(times)) * 1e3
    value = n / (ms / 1e3)
    line = {"impl": "reference", "metric": metric_name(args.config), "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "queries_per_step": n},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n} random queries per step, FP64 brute force over all {mesh.n_tris} triangles"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """Table 4 counterpart: each mesh built without and with site augmentation; list
    statistics (Max / Avg / Queried), query rate and build time.  One JSON line per build."""
    import torch
    import paper_2605_00429_gb300 as p2m
    from paper_2605_00429_gb300 import build as pbuild
    pbuild.build()
    torch.cuda.set_device(0)
    cases = [
        ("sphere: icosphere(5), 20,480 faces, no noise; 1M queries uniform in 1.2x bbox",
         lambda: (W.icosphere(5), None)),
        ("UV sphere 32x16, 960 faces; 1M queries uniform in 1.2x bbox", lambda: (W.uv_sphere(32, 16), None)),
        ("noisy sphere: icosphere(6) + noise, 81,920 faces; 1M queries as config 2",
         lambda: W.workload_large(1_000_000)),
        ("cylinder + cone 512x128, 203,776 faces; 1M queries as config 3",
         lambda: W.workload_symmetric(1_000_000)),
    ]
    # (label, build parameters): no augmentation, augmentation with the single Eq. 8 ball per
    # auxiliary site, augmentation with its per-corner balls (the default), and the same with
    # each centre site at its tau-cell's centre instead of its Voronoi vertices' centroid
    modes = [("off", dict(enable_aux=0)), ("on, Eq. 8 ball", dict(enable_aux=1, aux_balls=0)),
             ("on, corner balls", dict(enable_aux=1, aux_balls=1)),
             ("on, corner balls, p_c at the cell centre", dict(enable_aux=1, aux_balls=1, aux_centre=0))]
    for desc, make in cases:
        mesh, q = make()
        if q is None:
            q = W.queries_uniform_box(mesh, 1_000_000, 1.2, seed=1)
        pts = torch.from_numpy(q).cuda()
        for label, prm in modes:
            t0 = time.perf_counter()
            idx = p2m.P2MIndex(mesh.verts, mesh.tris, **prm)
            build_ms = (time.perf_counter() - t0) * 1e3
            st = idx.stats()
            c = idx.counters(pts)
            out = idx.query(pts)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                idx.query(pts, out=out)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            print(json.dumps({"ablation": desc, "aux": label, "build_ms": build_ms, "query_ms": ms,
                              "queries_per_s": len(q) / (ms / 1e3), "max_list": st["max_row"],
                              "avg_list": st["avg_row"], "queried_list": c["queried_list"] / len(q),
                              "queried_entries": c["row_entries"] / len(q),
                              "queried_exact": c["exact_tests"] / len(q), "long_queries": c["long_queries"],
                              "sites": st["n_sites"], "aux_sites": st["n_aux_sites"], "nnz": st["nnz"]}), flush=True)
            del idx


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--queries", type=int, default=0, help="override the workload's query count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip fwd+bwd and e2e legs")
    ap.add_argument("--schedule", type=int, default=5)
    ap.add_argument("--ablation", action="store_true", help="Table-4 style runs with / without site augmentation")
    ap.add_argument("--profile-range", action="store_true",
                    help="after the warm-up, run one query pass between cudaProfilerStart/Stop and exit "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.ablation:
        return run_ablation(args)
    args.warmup = max(args.warmup, 3)

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2605_00429_gb300 import build as pbuild
    if rank == 0 or world == 1:
        pbuild.build()
    barrier()
    import paper_2605_00429_gb300 as p2m

    desc, make = WORKLOADS[args.config]
    mesh, q = make(args.queries)
    n = q.shape[0]
    t0 = time.perf_counter()
    idx = p2m.P2MIndex(mesh.verts, mesh.tris, schedule=args.schedule)
    build_wall_ms = (time.perf_counter() - t0) * 1e3
    st = idx.stats()
    pts = torch.from_numpy(q).to(dev)
    out = (torch.empty(n, device=dev), torch.empty(n, 3, device=dev), torch.empty(n, device=dev, dtype=torch.int32),
           torch.empty(n, 3, device=dev))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    for _ in range(args.warmup):
        idx.query(pts, out=out)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
        idx.query(pts, out=out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_range": desc, "queries": n, "schedule": args.schedule}), flush=True)
        return

    # instrumented pass (untimed): work counters for the algorithmic FLOP count
    cnt = idx.counters(pts)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # the library records CUDA events on the query's stream around its list-scan kernel (the
    # dominant kernel); they are read after each step, outside the step's own events
    idx.set_timing(True)
    scan_ms = []
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        starts[k].record(stream)
        idx.query(pts, out=out)
        ends[k].record(stream)
        scan_ms.append(idx.query_timing()[0])
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    idx.set_timing(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = reduce_max_ms(float(np.mean(step_ms)), world, dev)
    kernel_ms = float(np.mean(scan_ms))
    value = replicas_value(n, ms, world)

    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    flops = (FLOP_PER_SITE * cnt["site_candidates"] + FLOP_PER_ROW_ENTRY * cnt["row_entries"] +
             FLOP_PER_EXACT * cnt["exact_tests"] + FLOP_PER_QUERY * n)
    # the list-scan kernel's own work: the short lists' entries and exact tests (the long lists'
    # belong to the warp pass) and its per-query bound setup and record
    scan_flops = (FLOP_PER_ROW_ENTRY * (cnt["row_entries"] - cnt["long_entries"]) +
                  FLOP_PER_EXACT * cnt["exact_tests"] + FLOP_PER_QUERY * n)
    achieved = scan_flops / (kernel_ms / 1e3) / 1e12 if kernel_ms > 0 else flops / (ms / 1e3) / 1e12
    hbm_gbs = BYTES_PER_QUERY * n / (ms / 1e3) / 1e9

    line = {"metric": metric_name(args.config), "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "queries": n, "tris": mesh.n_tris, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "gpu_launches": OWN_KERNELS_PER_STEP.get(args.schedule, 6) * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": profiled_traffic(args.config, n),
                         "l1tex_pct_ncu": profiled_l1tex_pct(args.config),
                         "kernel": "k_query_staged" if args.schedule == 5 else "k_query_thread",
                         "kernel_ms": kernel_ms,
                         "kernel_share_of_step": kernel_ms / ms if ms > 0 else None,
                         "step_flops_achieved": flops / (ms / 1e3) / 1e12,
                         "peak_kind": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x max SM clock "
                                      f"from {pk_kind} peaks",
                         "sm_count": sm_count,
                         "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": pk.get("hbm_gbs"),
                         "hbm_frac": hbm_gbs / float(pk.get("hbm_gbs", 6800.0))},
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "csr_build_ms": st["ms_tri"] + st["ms_lbvh"] + st["ms_k1"],
            "build": {"wall_ms": build_wall_ms, "host_delaunay_ms": st["ms_delaunay"], "host_aug_ms": st["ms_aug"],
                      "gpu_cells_ms": st["ms_cells"], "cells_clipped_on_host": st["n_cells_host"], "gpu_lists_ms": st["ms_k1"], "gpu_grid_ms": st["ms_grid"],
                      "sites": st["n_sites"], "aux_sites": st["n_aux_sites"], "nnz": st["nnz"],
                      "max_list": st["max_row"], "avg_list": st["avg_row"], "grid": st["grid_res"],
                      "grid_entries": st["grid_entries"], "grid_max": st["grid_max"]},
            "counters": {"queried_list": cnt["queried_list"] / n,
                         "queried_entries": cnt["row_entries"] / n, "queried_exact": cnt["exact_tests"] / n,
                         "sites_per_query": cnt["site_candidates"] / n, "outside": cnt["n_outside"],
                         "tie_rechecks": cnt["tie_rechecks"], "long_queries": cnt["long_queries"],
                         "long_entries_per_long_query": cnt["long_entries"] / max(1, cnt["long_queries"])}}

    if not args.no_extras:
        # end to end through the host-buffer C-ABI call: pinned inputs, all four outputs back
        hp = torch.from_numpy(q).pin_memory()
        hd = torch.empty(n, dtype=torch.float32).pin_memory()
        hc = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        ht = torch.empty(n, dtype=torch.int32).pin_memory()
        hb = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        idx.query_host(hp, hd, hc, ht, hb)
        e2e_steps = max(1, min(args.steps, 10))
        barrier()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            idx.query_host(hp, hd, hc, ht, hb)
        # every leg below is whole-job: N ranks' queries over the slowest rank's time
        e2e_s = reduce_max_ms((time.perf_counter() - t) / e2e_steps * 1e3, world, dev) / 1e3
        line["e2e"] = {"value": world * n / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": 12 * n,
                       "d2h_bytes_per_step": 32 * n}
        # fwd + bwd on the differentiation workload
        dm, dq = W.workload_diff(1_000_000)
        didx = p2m.P2MIndex(dm.verts, dm.tris)
        verts = torch.from_numpy(dm.verts).to(dev).requires_grad_(True)
        dpts = torch.from_numpy(dq).to(dev).requires_grad_(True)

        def fb():
            d = p2m.unsigned_distance(dpts, verts, didx)
            loss = (d * d).sum()
            loss.backward()
            return loss
        for _ in range(3):
            fb()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fsteps = max(3, min(args.steps, 20))
        e0.record()
        for _ in range(fsteps):
            verts.grad = None
            dpts.grad = None
            fb()
        e1.record()
        torch.cuda.synchronize()
        fb_ms = reduce_max_ms(e0.elapsed_time(e1) / fsteps, world, dev)
        line["fwd_bwd"] = {"value": world * dq.shape[0] / (fb_ms / 1e3), "unit": "queries/s", "ms_per_step": fb_ms,
                           "workload": WORKLOADS["diff"][0] + "; loss = sum d^2, grads to points and vertices"}
        # batching: 256 meshes behind one persistent launch (graph) vs one launch per mesh
        meshes, bq = W.workload_batch(256)
        bidx = p2m.P2MIndex.batch([(m_.verts, m_.tris) for m_ in meshes])
        boff = np.concatenate([[0], np.cumsum([len(x) for x in bq])]).astype(np.int64)
        bpts = torch.from_numpy(np.concatenate(bq)).to(dev)
        del bq
        nb = bpts.shape[0]
        bout = (torch.empty(nb, device=dev), torch.empty(nb, 3, device=dev),
                torch.empty(nb, device=dev, dtype=torch.int32), torch.empty(nb, 3, device=dev))
        res = {}
        for label, mode, graph in (("batched", 0, True), ("per_mesh", 1, False)):
            for _ in range(2):
                bidx.batch_query(bpts, boff, mode=mode, use_graph=graph, out=bout)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            bsteps = max(3, min(args.steps, 10))
            e0.record()
            for _ in range(bsteps):
                bidx.batch_query(bpts, boff, mode=mode, use_graph=graph, out=bout)
            e1.record()
            torch.cuda.synchronize()
            res[label] = reduce_max_ms(e0.elapsed_time(e1) / bsteps, world, dev)
        line["batch"] = {"value": world * nb / (res["batched"] / 1e3), "unit": "queries/s",
                         "ms_per_step": res["batched"],
                         "per_mesh_value": world * nb / (res["per_mesh"] / 1e3), "per_mesh_ms": res["per_mesh"],
                         "speedup": res["per_mesh"] / res["batched"], "queries": nb, "meshes": len(meshes),
                         "tris": int(sum(m_.n_tris for m_ in meshes)),
                         "workload": "256 noisy geodesic spheres / capped cylinders, T log-uniform [500, 200k], "
                                     "Q log-uniform [1k, 1M]; one persistent launch in a CUDA graph vs one launch per mesh"}
        del bidx, bpts, bout
        # the other workloads of the contract, each on its own index, and the forward alone on
        # the differentiation workload (beside fwd_bwd)
        legs = {}
        for key in ("small", "symmetric", "diff"):
            if key == args.config:
                continue
            legs["diff_forward" if key == "diff" else key] = config_leg(
                p2m, key, dev, max(3, min(args.steps, 20)), args.schedule, flush, float(pk.get("hbm_gbs", 6800.0)))
        line["configs"] = legs
    else:
        line["e2e"] = None

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mesh, q)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
