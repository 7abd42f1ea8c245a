#!/usr/bin/env python
"""Exact-DPC throughput on GB300: points/s for rho + lambda/delta + labels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1|c4|c5]
                    [--precision fp32|fp64] [--impl ours|reference]

The default workload is c3: 1e7 points in 3-D (the seed-spreader set), the
size at which the float32-certified path is compared with the plain binary64
path.

One step is one ``dpc_run`` call: binning, density, dependent points and
labels for every cutoff of the workload, inputs resident in HBM, timed with
CUDA events on the launching stream; L2 is flushed (a 512 MiB write) between
steps, outside the timed events.  ``value`` = points x cutoffs / second over
the K timed steps, summed over ranks (each rank runs an independent replica:
the method has no cross-point-set exchange, so N > 1 is replicas only).

Extra keys: ``fp64_path`` (same workload with every distance in binary64),
``e2e`` (dpc_run_host: pinned host buffers, copies inside the timed region),
``roofline`` (the dominant kernel, against the FFMA rate measured in the same
run), ``peaks`` (measured FFMA and DFMA rates), ``cpu_baseline`` (the exact
kd-tree CPU oracle on the same workload, all host cores), ``clocks``,
``phases_ms``.

``--impl reference`` times the CPU oracle alone (the paper publishes no code
that runs here; the oracle is the reference arm), on rank 0: each step is one
full run of the kd-tree oracle on the workload (rho, lambda, delta at every
cutoff, labels omitted), as many steps as fit in about two minutes.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "exact-DPC points/s (rho+delta+labels), FP32-certified vs FP64 path, 1 GB300"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")

# FP32 issue peak derived from unit counts and clocks, for comparison with
# the measured one: SMs x 128 FP32 lanes x 2 flops per FMA x max SM clock.
FP32_LANES = 128
LAYOUT_NAMES = ["?", "union", "segment", "tree", "tensor", "pairs", "cell"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5", "spreader"],
                    help="spreader: the seed-spreader family of c3 at --n points in --d dimensions "
                         "(reduced cases for profiling)")
    ap.add_argument("--n", type=int, default=4_000_000, help="points of --workload spreader")
    ap.add_argument("--d", type=int, default=3, help="dimension of --workload spreader")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fast", action="store_true", help="skip the fp64, e2e and CPU legs (profiling runs)")
    ap.add_argument("--cpu-instances", type=int, default=96,
                    help="batched workload: instances the CPU oracle baseline runs (a seeded sample)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default grid-level rule")
    ap.add_argument("--no-graph", action="store_true", help="time plain calls instead of graph replays")
    ap.add_argument("--layout", default="auto", choices=["auto", "union", "segment", "tree", "tensor", "pairs", "cell"],
                    help="fixed kernel layout (auto: the autotuned choice)")
    ap.add_argument("--near-shift", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="fixed near-phase grid level below the density's (-1: the autotuned choice)")
    ap.add_argument("--study", default="none", choices=["none", "scaling", "dcut", "next"],
                    help="scaling: time over n = 1e3..1e7 on the seed-spreader family in 2-D and 3-D; "
                         "dcut: phase times over a d_cut sweep on c2 and c3; next: the decision-graph "
                         "summaries and the priority range search on c3 and c4 (one JSON line per point)")
    return ap.parse_args()


def load_workload(name, n=4_000_000, d=3):
    if name == "spreader":
        return W.spreader(n, d)
    return {"c1": W.c1, "c2": W.c2, "c3": W.c3, "c4": W.c4, "c5": W.c5}[name]()


class Job:
    """One workload as the library sees it: packed coordinates, the batch
    descriptor arguments and the thresholds (single point sets are batches of
    one instance)."""

    def __init__(self, w):
        self.w = w
        self.name = w.name
        if isinstance(w, W.BatchWorkload):
            self.flat = w.flat
            self.sizes, self.dims, self.coord_offset = list(w.sizes), list(w.dims), list(w.coord_offset)
            self.d_cut = [list(r) for r in w.d_cut]
        else:
            self.flat = w.pts
            self.sizes, self.dims, self.coord_offset = [w.n], [w.d], [0]
            self.d_cut = [list(w.d_cut)]
        self.rho_noise, self.rho_min, self.delta_min = w.rho_noise, w.rho_min, w.delta_min
        self.n_dcut = len(self.d_cut[0])
        self.N = int(sum(self.sizes))
        self.pt_offset = [0]
        for n in self.sizes:
            self.pt_offset.append(self.pt_offset[-1] + n)

    def instance(self, i):
        o = self.coord_offset[i]
        return np.asarray(self.flat[o:o + self.sizes[i] * self.dims[i]]).reshape(self.sizes[i], self.dims[i])

    def config(self):
        if len(self.sizes) == 1:
            return {"workload": self.name, "n": self.N, "d": self.dims[0], "d_cut": self.d_cut[0],
                    "rho_noise": self.rho_noise, "rho_min": self.rho_min, "delta_min": self.delta_min}
        return {"workload": self.name, "instances": len(self.sizes), "points": self.N,
                "d_counts": {str(d): self.dims.count(d) for d in sorted(set(self.dims))},
                "n_range": [min(self.sizes), max(self.sizes)], "d_cuts_per_instance": self.n_dcut,
                "thresholds": "per (instance, cutoff): rho_noise = rho_min = 2 x median rho, "
                              "delta_min = 5 d_cut"}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CPU oracle on a bounded sample


def cpu_oracle_run(job, max_instances, seed):
    """The exact kd-tree CPU oracle (oracle.tree_run / tree_batch: rho, lambda
    and delta of every point at every cutoff; labels omitted, they are O(n))
    on the workload, all host cores.  A single point set runs whole; a batch
    runs a seeded sample of ``max_instances`` instances.  Returns (points x
    cutoffs / s, seconds, threads, description of the sample)."""
    import oracle
    t0 = time.perf_counter()
    if len(job.sizes) == 1:
        oracle.tree_run(job.instance(0), job.d_cut[0])
        units = job.N * job.n_dcut
        what = "the whole %s (%d points x %d cutoffs)" % (job.name, job.N, job.n_dcut)
    else:
        rng = np.random.default_rng(seed)
        ids = np.sort(rng.choice(len(job.sizes), size=min(max_instances, len(job.sizes)), replace=False))
        parts = [job.instance(int(i)).reshape(-1) for i in ids]
        flat = np.concatenate(parts)
        po = np.concatenate([[0], np.cumsum([job.sizes[int(i)] for i in ids])]).astype(np.int64)
        co = np.concatenate([[0], np.cumsum([p.size for p in parts])[:-1]]).astype(np.int64)
        t0 = time.perf_counter()
        oracle.tree_batch(flat, po, co, [job.dims[int(i)] for i in ids], [job.d_cut[int(i)] for i in ids])
        units = int(po[-1]) * job.n_dcut
        what = "%d seeded instances of %s (%d points) x %d cutoffs" % (len(ids), job.name, int(po[-1]),
                                                                       job.n_dcut)
    dt = time.perf_counter() - t0
    return units / dt, dt, oracle.threads(), what


# ---------------------------------------------------------------------------
# roofline of the search kernels


def ball_volume(d):
    return math.pi ** (d / 2.0) / math.gamma(d / 2.0 + 1.0)


def block_work(job, rho_dev):
    """Algorithmic flops of the density (or near-dependent) launches of one
    step, summed over instances and cutoffs: per point, the candidates of the
    3^d block of grid cells of side d_cut around it, rho * 3^d / V_d (V_d the
    volume of the unit d-ball), each d subtractions and d multiply-adds
    (3d flops).  For d > 3 this counts the candidates of an ideal grid over all
    d coordinates, fewer than the library's 3-coordinate grid visits."""
    import torch
    po = torch.tensor(job.pt_offset, dtype=torch.int64, device=rho_dev.device)
    factor = torch.tensor([3.0 ** d / ball_volume(d) * 3 * d for d in job.dims], dtype=torch.float64,
                          device=rho_dev.device)
    total = 0.0
    for c in range(rho_dev.shape[0]):
        cs = torch.cumsum(rho_dev[c].to(torch.float64), 0)
        cs = torch.cat([torch.zeros(1, dtype=torch.float64, device=cs.device), cs])
        per = cs[po[1:]] - cs[po[:-1]]
        total += float((per * factor).sum().item())
    mean_rho = float(rho_dev[0].to(torch.float64).mean().item()) if job.N else 0.0
    return total, mean_rho


def phase_rooflines(job, stats, phase_ms, hbm_gbs, peak_kind):
    """HBM rooflines of the two streaming phases of one step, from their
    algorithmic bytes per point and cutoff:
      binning  bbox (read the coordinates), keys (read them, write a 64-bit key
               and a 32-bit id), radix sort (one 8-byte read for the digit
               counts, then 24 bytes read and written per pass), gather (read
               the id and the coordinates, write the padded float point, key
               and id): 12 d + 48 + 24 passes + 4 DP bytes per point;
      labels   read rho, lambda and delta, write the label: 20 bytes per point
               and cutoff.
    Single point sets only (a batch mixes dimensions and pass counts)."""
    if len(job.sizes) != 1 or not phase_ms:
        return None
    d = job.dims[0]
    g = min(d, 4)
    dp = 2 if d <= 2 else (4 if d <= 4 else 8)
    passes = (g * int(stats.get("bits_per_axis", 0)) + 7) // 8
    out = {}
    for name, per_pt in (("bin", 12 * d + 48 + 24 * passes + 4 * dp), ("labels", 20 * job.n_dcut)):
        ms = phase_ms.get(name)
        if not ms:
            continue
        gbs = per_pt * job.N / (ms / 1e3) / 1e9
        out[name] = {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                     "bytes_per_point": per_pt, "ms": ms, "peak_source": peak_kind,
                     "passes": passes if name == "bin" else None}
    return out


def combine_ranks(total_ms, units_per_rank, steps, world, device=None):
    """Whole-job timing over replicas: the slowest rank's time bounds the job.
    Returns (max total ms over ranks, points/s of all ranks together)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, units_per_rank * world * steps / (total_ms / 1e3)


def load_traffic(kernel, workload):
    try:
        with open(TRAFFIC_PATH) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(kernel, {}).get(workload)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    try:
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return e["bytes_per_launch"] if sha == e.get("source_sha") else None


# ---------------------------------------------------------------------------


def run_ours(args, rank, world, dev):
    import torch
    import paper_2305_11335_gb300 as dpc
    from paper_2305_11335_gb300 import _build

    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    job = Job(load_workload(args.workload, args.n, args.d))
    batch = dpc.Batch(job.pt_offset, job.dims, job.d_cut, coord_offset=job.coord_offset)
    params = dpc.make_params(batch, job.rho_noise, job.rho_min, job.delta_min)
    # one stream for every call (the library keeps one workspace, autotuning
    # cache and captured graph per stream); graph capture needs a stream other
    # than the legacy default one
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    pts = torch.from_numpy(job.flat).to(dev)
    shape = (batch.n_dcut, job.N)
    out = {"rho": torch.empty(shape, dtype=torch.int32, device=dev),
           "lam": torch.empty(shape, dtype=torch.int32, device=dev),
           "delta": torch.empty(shape, dtype=torch.float64, device=dev),
           "label": torch.empty(shape, dtype=torch.int32, device=dev)}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    units = job.N * batch.n_dcut

    def timed_steps(k, precision, phase_times, graph=False):
        times, phases = [], {}
        for _ in range(k):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dpc.dpc_run(pts, batch, params, precision=precision, stream=stream, out=out, phase_times=phase_times,
                        graph=graph, layout=args.layout, near_shift=args.near_shift)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            if phase_times:
                for p, (ms, cnt) in dpc.dpc_get_phase_times(stream).items():
                    acc = phases.setdefault(p, [0.0, 0])
                    acc[0] += ms
                    acc[1] += cnt
        return times, phases

    # warm-up: at least W steps and about a second of load (for the clock record)
    sampler = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    if sampler:
        sampler.start()
    t_end = time.time() + (0.0 if args.fast else 1.0)
    steps = 0
    while steps < args.warmup or time.time() < t_end:
        # the first warm-up call autotunes the grid level (cached for the rest)
        dpc.dpc_run(pts, batch, params, precision=args.precision, stream=stream, out=out, layout=args.layout,
                    near_shift=args.near_shift,
                    autotune=(steps == 0 and not args.no_autotune and args.layout == "auto"
                              and args.near_shift < 0))
        steps += 1
    use_graph = not args.no_graph
    # capture (graph mode) or one more plain call, then synchronize
    dpc.dpc_run(pts, batch, params, precision=args.precision, stream=stream, out=out, sync=True, graph=use_graph,
                layout=args.layout, near_shift=args.near_shift)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, _ = timed_steps(args.steps, args.precision, False, graph=use_graph)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    stats = dpc.dpc_get_stats(stream)
    # roofline denominators, measured on this GPU right after the timed steps
    fp32_peak = dpc.probe_peak("fp32", stream=stream)
    fp64_peak = dpc.probe_peak("fp64", stream=stream)
    # phase breakdown: a separate pass of plain (non-graph) calls with events
    # around every phase on the same stream
    k_ph = max(1, min(args.steps, 5))
    _, phases = timed_steps(k_ph, args.precision, True)
    phase_steps = k_ph
    total_ms, value = combine_ranks(sum(times), units, args.steps, world, dev)
    ms_per_step = total_ms / args.steps

    config = job.config()
    config.update({"precision": args.precision, "l2": "flushed between steps (512 MiB write)",
                   "grid_level": "autotuned in the first warm-up call" if not args.no_autotune else "default rule",
                   "block_radius": int(stats.get("block_radius", 0)),
                   "near_shift": int(stats.get("near_shift", 0)),
                   "layouts": {"density": LAYOUT_NAMES[int(stats.get("density_layout", 0))],
                               "near": LAYOUT_NAMES[int(stats.get("near_layout", 0))]},
                   "parallelism": "replicas" if world > 1 else "1 GPU"})
    res = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 filter + f64 recheck" if args.precision == "fp32" else "f64",
           "data": "synthetic (seeded generator standing in for the paper's data sets)",
           "config": config,
           "gpu_launches": int(stats["kernel_launches"]) * args.steps,
           "launch": ("one CUDA graph per step (DPC_FLAG_GRAPH: %d kernels captured once, replayed)"
                      % int(stats["kernel_launches"])) if use_graph else "one launch per kernel",
           "phases_ms": {p: round(v[0] / phase_steps, 5) for p, v in phases.items()},
           "phases_from": "%d plain calls with events around every phase, after the timed steps" % phase_steps,
           "stats": {k: int(v) for k, v in stats.items()}}
    if rank != 0:
        return None

    # roofline of the dominant kernel (density or near-dependent, whichever
    # takes longer): algorithmic flops per launch / CUDA-event time per launch
    pk, pk_kind = peaks()
    single = {p: v for p, v in phases.items() if p in ("density", "near", "far", "tree", "maxkey")}
    dom = max(single, key=lambda p: single[p][0]) if single else None
    kernels = {"density": {2: "k_density_seg", 4: "k_density_tc", 5: "k_density_pairs", 6: "k_density_cell"}.get(
        stats.get("density_layout"), "k_density"),
               "near": {2: "k_dep_near_seg", 3: "k_near_to_far", 6: "k_dep_near_cell"}.get(stats.get("near_layout"),
                                                                                          "k_dep_near")}
    model_phase = dom if dom in kernels else max(("density", "near"), key=lambda p: phases[p][0])
    work, mean_rho = block_work(job, out["rho"])
    high_d = max(job.dims) > 3
    if high_d:
        # the ideal all-coordinate grid overestimates clustered data above
        # 3 dimensions: count the pairs the density step actually scanned
        d_mean = float(np.dot(job.sizes, job.dims)) / max(1, job.N)
        work = float(stats.get("density_pairs", 0)) * 3.0 * d_mean
    pairs_layout = model_phase == "density" and int(stats.get("density_layout", 0)) == 5
    if pairs_layout and not high_d:
        work *= 0.5  # the pair layout evaluates each unordered pair once
    # phases[] holds the sums over the phase pass; work is one step's
    launches = phases[model_phase][1] // phase_steps
    step_ms = phases[model_phase][0] / phase_steps
    per_launch_ms = step_ms / launches
    achieved = work / (step_ms / 1e3) / 1e12
    clk = pk.get("sm_max_mhz", 2070.0)
    derived = torch.cuda.get_device_properties(dev).multi_processor_count * FP32_LANES * 2 * clk * 1e6 / 1e12
    peak = fp32_peak / 1e12
    res["peaks"] = {"fp32_tflops": fp32_peak / 1e12, "fp64_tflops": fp64_peak / 1e12,
                    "source": "measured in this run (dpc_probe_peak: FFMA / DFMA loops, CUDA events, clocks as "
                              "found)", "fp32_tflops_derived": derived}
    res["roofline"] = {
        "bound": "alu", "kernel": kernels[model_phase], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak, "traffic": load_traffic(kernels[model_phase], job.name),
        "peak_source": "measured: FFMA loop in this run (dpc_probe_peak), %.1f TFLOP/s; derived from unit "
                       "counts and the %.0f MHz max clock: %.1f" % (peak, clk, derived),
        "work": ("%.4g flops per step over %d launches: the %d (query, candidate) pairs the density step "
                 "scanned x 3d flops (d > 3: the ideal-grid count rho x 3^d / V_d overestimates clustered "
                 "data)" % (work, launches, int(stats.get("density_pairs", 0)))) if high_d else
                ("%.4g flops per step over %d launches: per point rho x 3^d / V_d block candidates x 3d flops "
                 "(mean rho %.1f at the first cutoff)%s" % (work, launches, mean_rho,
                                                             ", halved: each unordered pair once"
                                                             if pairs_layout else "")),
        "ms_per_launch": per_launch_ms}
    res["dominant_phase"] = dom
    res["phase_rooflines"] = phase_rooflines(job, stats, res["phases_ms"], pk.get("hbm_gbs", 6800.0),
                                             "measured" if pk_kind == "measured" else "fallback")

    if not args.fast:
        # the plain FP64 path on the same workload (binary64 costs 10-50x more
        # here; a workload whose FP32 step already takes over a second is left
        # out rather than holding the GPU for minutes)
        other = "fp64" if args.precision == "fp32" else "fp32"
        if other == "fp32" or ms_per_step < 1000.0:
            dpc.dpc_run(pts, batch, params, precision=other, stream=stream, out=out, sync=True)
            k2 = max(1, min(max(3, args.steps // 3), int(20000.0 / max(1.0, ms_per_step * 20))))
            t2, _ = timed_steps(k2, other, False)
            res[other + "_path"] = {"value": units * k2 / (sum(t2) / 1e3), "ms_per_step": sum(t2) / k2,
                                    "steps": k2}
        else:
            res[other + "_path"] = {"value": None, "skipped": "FP32 step %.0f ms; the binary64 path would take "
                                                             "minutes per step" % ms_per_step}
        # end to end through the host-buffer entry point
        hp = torch.from_numpy(job.flat).pin_memory()
        hout = {"rho": torch.empty(shape, dtype=torch.int32).pin_memory(),
                "lam": torch.empty(shape, dtype=torch.int32).pin_memory(),
                "delta": torch.empty(shape, dtype=torch.float64).pin_memory(),
                "label": torch.empty(shape, dtype=torch.int32).pin_memory()}
        dpc.dpc_run_host(hp, batch, params, precision=args.precision, stream=stream, out=hout)
        te = []
        for _ in range(max(3, args.steps // 3)):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dpc.dpc_run_host(hp, batch, params, precision=args.precision, stream=stream, out=hout)
            b.record(stream)
            b.synchronize()
            te.append(a.elapsed_time(b))
        res["e2e"] = {"value": units / (statistics.mean(te) / 1e3), "unit": "points/s",
                      "ms_per_step": statistics.mean(te), "h2d_bytes_per_step": int(job.flat.nbytes),
                      "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in hout.values())),
                      "api": "dpc_run_host"}
        # the exact CPU oracle on the same workload
        v, dt, th, what = cpu_oracle_run(job, args.cpu_instances, 99)
        res["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": th, "kind": "oracle",
                               "sample": "kd-tree oracle (rho, lambda, delta from the definitions; labels "
                                         "omitted) on %s, %.1f s wall" % (what, dt)}
    res["clocks"] = clocks
    return res


# ---------------------------------------------------------------------------
# studies (not the bench line): running time against n and against d_cut


def _study_point(dpc, torch, dev, stream, flush, w, steps, warmup, skip_noise=False):
    """Median graph-replay time of dpc_run on workload ``w`` (one cutoff),
    the phase times of one plain call, and the mean density."""
    job = Job(w)
    batch = dpc.Batch(job.pt_offset, job.dims, job.d_cut, coord_offset=job.coord_offset)
    params = dpc.make_params(batch, job.rho_noise, job.rho_min, job.delta_min)
    pts = torch.from_numpy(job.flat).to(dev)
    shape = (batch.n_dcut, job.N)
    out = {"rho": torch.empty(shape, dtype=torch.int32, device=dev),
           "lam": torch.empty(shape, dtype=torch.int32, device=dev),
           "delta": torch.empty(shape, dtype=torch.float64, device=dev),
           "label": torch.empty(shape, dtype=torch.int32, device=dev)}
    for i in range(max(3, warmup)):
        dpc.dpc_run(pts, batch, params, stream=stream, out=out, autotune=(i == 0), skip_noise=skip_noise)
    dpc.dpc_run(pts, batch, params, stream=stream, out=out, sync=True, graph=True, skip_noise=skip_noise)
    times = []
    for _ in range(steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dpc.dpc_run(pts, batch, params, stream=stream, out=out, graph=True, skip_noise=skip_noise)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    dpc.dpc_run(pts, batch, params, stream=stream, out=out, sync=True, phase_times=True, skip_noise=skip_noise)
    ph = {p: round(v[0], 5) for p, v in dpc.dpc_get_phase_times(stream).items()}
    rho = out["rho"][0].double()
    mean_rho = float(rho.mean()) if job.N else 0.0
    noise = float((out["rho"][0] < int(job.rho_noise[0])).double().mean()) if job.N else 0.0
    del pts, out
    return job, statistics.median(times), ph, mean_rho, noise


def run_study(args, dev):
    import torch
    import paper_2305_11335_gb300 as dpc
    from paper_2305_11335_gb300 import _build

    _build.build()
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(3, args.steps)
    if args.study == "scaling":
        # Section 7's scalability over n (1e3..1e7), d_cut = 30, rho_min = 0,
        # delta_min = 100, on the seed-spreader family (2-D stands in for simden)
        for d in (2, 3):
            ns, ms = [], []
            for e in range(3, 8):
                n = 10 ** e
                job, t, ph, mean_rho, _ = _study_point(dpc, torch, dev, stream, flush, W.spreader(n, d), steps,
                                                       args.warmup)
                ns.append(n)
                ms.append(t)
                print(json.dumps({"study": "scaling", "workload": job.name, "n": n, "d": d, "ms": t,
                                  "points_per_s": n / (t / 1e3), "mean_rho": mean_rho, "phases_ms": ph}),
                      flush=True)
            x, y = np.log10(ns), np.log10(ms)
            print(json.dumps({"study": "scaling", "d": d, "summary": True,
                              "slope_log_time_vs_log_n": float(np.polyfit(x, y, 1)[0]),
                              "slope_n_ge_1e5": float(np.polyfit(x[2:], y[2:], 1)[0]),
                              "paper_slope_dpc_priority": 0.94}), flush=True)
    elif args.study == "next":
        run_next(args, dev, dpc, torch, stream, flush, steps)
    else:
        # the d_cut study (the paper's appendix on d_cut): with the noise
        # threshold fixed, sweep d_cut and split the time into density and
        # dependent-point finding; noise points skip the dependent search
        for name in ("c2", "c3"):
            base = load_workload(name)
            for f in (0.25, 0.5, 1.0, 2.0, 4.0):
                w = W.Workload(base.name, base.pts, [base.d_cut[0] * f], base.rho_noise[:1], base.rho_min[:1],
                               base.delta_min[:1])
                job, t, ph, mean_rho, noise = _study_point(dpc, torch, dev, stream, flush, w, steps,
                                                           args.warmup, skip_noise=True)
                dep = ph["maxkey"] + ph["near"] + ph["far"]
                print(json.dumps({"study": "dcut", "workload": base.name, "d_cut": base.d_cut[0] * f,
                                  "d_cut_factor": f, "avg_pct_within_d_cut": 100.0 * mean_rho / job.N,
                                  "mean_rho": mean_rho, "noise_fraction": noise, "rho_noise": int(job.rho_noise[0]),
                                  "ms": t, "density_ms": ph["density"], "dependent_ms": dep,
                                  "phases_ms": ph}), flush=True)


def _events_ms(torch, stream, flush, fn, steps):
    """Median CUDA-event time of fn() on `stream` (L2 flushed before each)."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def run_next(args, dev, dpc, torch, stream, flush, steps):
    """Throughput of the decision-graph summaries and the priority range
    search on the outputs of a full run (c3: one 1e7-point set; c4: the
    4096-instance batch, first cutoff)."""
    pk, pk_kind = peaks()
    for name in ("c3", "c4"):
        job = Job(load_workload(name))
        batch = dpc.Batch(job.pt_offset, job.dims, job.d_cut, coord_offset=job.coord_offset)
        params = dpc.make_params(batch, job.rho_noise, job.rho_min, job.delta_min)
        pts = torch.from_numpy(job.flat).to(dev)
        out = dpc.dpc_run(pts, batch, params, stream=stream, sync=True)
        rho, delta = out["rho"][0].contiguous(), out["delta"][0].contiguous()
        for k, rb, db in ((16, 0, 0), (1024, 0, 0), (0, 24, 48)):
            ms = _events_ms(torch, stream, flush, lambda: dpc.dpc_decision_graph(
                batch, rho, delta, k=k, rho_bins=rb, delta_bins=db, delta_lo=1e-3 * job.d_cut[0][0],
                stream=stream), steps)
            nbytes = 12.0 * job.N  # rho + delta read once: the algorithmic minimum
            gbs = nbytes / (ms / 1e3) / 1e9
            print(json.dumps({"study": "next", "op": "dpc_decision_graph", "workload": job.name,
                              "k": k, "rho_bins": rb, "delta_bins": db, "points": job.N, "ms": ms,
                              "points_per_s": job.N / (ms / 1e3),
                              "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"],
                                           "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                                           "peak_source": pk_kind,
                                           "work": "12 B per point (rho, delta read once)"}}), flush=True)
        # priority range: boxes of 2 d_cut around random points, threshold = the
        # point's own density (the points that could be its dependent point)
        rng = np.random.default_rng(7)
        nq = 100_000
        rows = rng.integers(0, len(job.sizes), nq)
        rows = rows[np.asarray(job.sizes)[rows] > 0]
        nq = len(rows)
        lo = np.zeros((nq, 8))
        hi = np.zeros((nq, 8))
        rq = np.zeros(nq, np.int32)
        rho_h = rho.cpu().numpy()
        for t, r in enumerate(rows.tolist()):
            j = int(rng.integers(0, job.sizes[r]))
            x = job.instance(r)[j].astype(np.float64)
            w = 2.0 * job.d_cut[r][0]
            lo[t, :len(x)], hi[t, :len(x)] = x - w, x + w
            rq[t] = rho_h[job.pt_offset[r] + j]
        q_inst = torch.from_numpy(rows.astype(np.int32)).to(dev)
        box = torch.from_numpy(np.stack([lo, hi], axis=1)).to(dev)
        q_rho = torch.from_numpy(rq).to(dev)
        for max_out in (0, 64):
            res = {}

            def call():
                res["o"] = dpc.dpc_priority_range(pts, batch, rho, q_inst, box, q_rho, max_out=max_out,
                                                  stream=stream)
            ms = _events_ms(torch, stream, flush, call, steps)
            cnt = res["o"]["count"].double()
            print(json.dumps({"study": "next", "op": "dpc_priority_range", "workload": job.name,
                              "queries": nq, "max_out": max_out, "ms": ms, "queries_per_s": nq / (ms / 1e3),
                              "mean_matches": float(cnt.mean()), "box": "2 d_cut half-width around a point",
                              "threshold": "the point's own density",
                              "includes": "binning and tree of every class (the call builds them)"}),
                  flush=True)
        del pts, out, rho, delta


def run_reference(args, rank, world):
    """The reference arm: the exact kd-tree CPU oracle on this workload, one
    full run per step (a batch: the seeded instance sample), as many timed
    steps as fit in about two minutes after one warm-up run."""
    if rank != 0:
        return None
    job = Job(load_workload(args.workload, args.n, args.d))
    warm = min(1, args.warmup)
    for s in range(warm):
        cpu_oracle_run(job, args.cpu_instances, 99)
    secs, vals = [], []
    th, what = 1, ""
    budget = 120.0
    while len(secs) < args.steps and (not secs or sum(secs) + secs[-1] <= budget):
        v, dt, th, what = cpu_oracle_run(job, args.cpu_instances, 99)
        secs.append(dt)
        vals.append(v)
    units = vals[0] * secs[0]
    value = units * len(secs) / sum(secs)
    ms = 1e3 * sum(secs) / len(secs)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": len(secs), "steps_requested": args.steps, "warmup": warm, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": job.config(),
            "cpu_baseline": {"kind": "oracle", "cores": th, "value": value,
                             "sample": "kd-tree oracle on %s per step (rho, lambda, delta from the definitions; "
                                       "labels omitted); steps capped at about %d s in total" % (what, budget)},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    if args.study != "none":
        if world > 1:
            raise SystemExit("--study runs on one GPU")
        run_study(args, dev)
        return
    res = run_ours(args, rank, world, dev)
    if res is not None:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
