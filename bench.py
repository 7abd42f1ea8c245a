#!/usr/bin/env python
"""Exact-DPC throughput on GB300: points/s for rho + lambda/delta + labels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2|c3|c1|c5]
                    [--precision fp32|fp64] [--impl ours|reference]

One step is one ``dpc_run`` call: binning, density, dependent points and
labels for every cutoff of the workload, inputs resident in HBM, timed with
CUDA events on the launching stream; L2 is flushed (a 512 MiB write) between
steps, outside the timed events.  ``value`` = points x cutoffs / second over
the K timed steps, summed over ranks (each rank runs an independent replica:
the method has no cross-point-set exchange, so N > 1 is replicas only).

Extra keys: ``fp64_path`` (same workload with every distance in binary64),
``e2e`` (dpc_run_host: pinned host buffers, copies inside the timed region),
``roofline`` (the dominant kernel), ``cpu_baseline`` (the CPU oracle on a
bounded sample of the same workload), ``clocks``, ``phases_ms``.

``--impl reference`` times the CPU oracle alone (the paper publishes no code
that runs here; the oracle is the reference arm), on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

# FP32 issue peak derived from unit counts and clocks: 152 SMs x 128 FP32
# lanes x 2 flops per FMA x max SM clock.
SMS = 152
FP32_LANES = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c5"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fast", action="store_true", help="skip the fp64, e2e and CPU legs (profiling runs)")
    ap.add_argument("--cpu-sample", type=int, default=4096)
    return ap.parse_args()


def load_workload(name):
    return {"c1": W.c1, "c2": W.c2, "c3": W.c3, "c5": W.c5}[name]()


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


def cpu_oracle_sample(pts, d_cuts, m, seed):
    """rho, lambda and delta of m seeded sample points of the full workload,
    evaluated from the definitions by the oracle.  Returns (points/s, seconds,
    threads)."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(pts.shape[0], size=min(m, pts.shape[0]), replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    for dc in d_cuts:
        oracle.density(pts, dc, idx=idx)
        oracle.dependent_at(pts, dc, idx, max_checks=256)
    dt = time.perf_counter() - t0
    return len(idx) * len(d_cuts) / dt, dt, oracle.threads()


# ---------------------------------------------------------------------------
# roofline of one phase

def phase_model(phase, w, out_rho):
    """Algorithmic work of one launch of the density or near-dependent kernel:
    per point the candidates of the 3^g block of cells of side d_cut, each
    d subtractions and d multiply-adds (3d flops).  Defined for d <= 3, where
    the grid covers every coordinate."""
    n, d = w.n, w.d
    g = min(d, 3)
    if d > 3:
        return None, None, None, ""
    if phase == "density":
        # candidates of the 3^g block at cell side d_cut per point:
        # rho * 3^g / V_g (V_g = volume of the unit ball in g dims, times 2^g / 2^g),
        # each d subtractions and d FMAs = 3d flops
        vol = {1: 2.0, 2: np.pi, 3: 4.0 / 3.0 * np.pi}[g]
        cand = float(out_rho.astype(np.float64).mean()) * (3.0 ** g) / vol
        flops = n * cand * 3 * d
        return "alu", flops, "TFLOP/s", "%d points x %.1f block candidates x %d flops" % (n, cand, 3 * d)
    return None, None, None, ""


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
    w = load_workload(args.workload)
    n, d = w.n, w.d
    batch = dpc.Batch.single(n, d, w.d_cut)
    params = dpc.make_params(batch, w.rho_noise, w.rho_min, w.delta_min)
    stream = torch.cuda.current_stream()
    pts = torch.from_numpy(w.pts).to(dev)
    shape = (batch.n_dcut, n)
    out = {"rho": torch.empty(shape, dtype=torch.int32, device=dev),
           "lam": torch.empty(shape, dtype=torch.int32, device=dev),
           "delta": torch.empty(shape, dtype=torch.float64, device=dev),
           "label": torch.empty(shape, dtype=torch.int32, device=dev)}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    units = n * batch.n_dcut

    def timed_steps(k, precision, phase_times):
        times, phases = [], {}
        for _ in range(k):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dpc.dpc_run(pts, batch, params, precision=precision, stream=stream, out=out, phase_times=phase_times)
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
        dpc.dpc_run(pts, batch, params, precision=args.precision, stream=stream, out=out)
        steps += 1
    dpc.dpc_run(pts, batch, params, precision=args.precision, stream=stream, out=out, sync=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, phases = timed_steps(args.steps, args.precision, True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    stats = dpc.dpc_get_stats(stream)
    total_ms, value = combine_ranks(sum(times), units, args.steps, world, dev)
    ms_per_step = total_ms / args.steps

    res = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 filter + f64 recheck" if args.precision == "fp32" else "f64",
           "data": "synthetic (seeded generator standing in for the paper's data sets)",
           "config": {"workload": w.name, "n": n, "d": d, "d_cut": w.d_cut, "rho_noise": w.rho_noise,
                      "rho_min": w.rho_min, "delta_min": w.delta_min, "precision": args.precision,
                      "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
           "gpu_launches": int(stats["kernel_launches"]) * args.steps,
           "phases_ms": {p: round(v[0] / args.steps, 5) for p, v in phases.items()},
           "stats": {k: int(v) for k, v in stats.items()}}
    if rank != 0:
        return None

    # roofline of the dominant kernel: the longest single-launch phase
    rho_host = out["rho"].cpu().numpy()
    pk, pk_kind = peaks()
    single = {p: v for p, v in phases.items() if p in ("density", "near", "far", "tree", "maxkey")}
    dom = max(single, key=lambda p: single[p][0]) if single else None
    roof = None
    kernels = {"density": "k_density", "near": "k_dep_near"}
    model_phase = dom if dom in kernels else max(("density", "near"), key=lambda p: phases[p][0])
    bound, work, unit, how = phase_model("density", w, rho_host)
    if work is not None:
        per_launch_ms = phases[model_phase][0] / phases[model_phase][1]
        achieved = work / (per_launch_ms / 1e3) / 1e12
        clk = pk.get("sm_max_mhz", 2070.0)
        peak = SMS * FP32_LANES * 2 * clk * 1e6 / 1e12
        roof = {"bound": bound, "kernel": kernels[model_phase], "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak,
                "traffic": load_traffic(kernels[model_phase], w.name),
                "peak_source": "derived (no FP32 figure is measured): 152 SMs x 128 FP32 lanes x 2 flops x "
                               "%.0f MHz max SM clock" % clk,
                "work": how, "ms_per_launch": per_launch_ms}
    res["roofline"] = roof
    res["dominant_phase"] = dom

    if not args.fast:
        # the plain FP64 path on the same workload
        other = "fp64" if args.precision == "fp32" else "fp32"
        dpc.dpc_run(pts, batch, params, precision=other, stream=stream, out=out, sync=True)
        k2 = max(3, args.steps // 3)
        t2, _ = timed_steps(k2, other, False)
        res[other + "_path"] = {"value": units * k2 / (sum(t2) / 1e3), "ms_per_step": sum(t2) / k2,
                                "steps": k2}
        # end to end through the host-buffer entry point
        hp = torch.from_numpy(w.pts).pin_memory()
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
                      "ms_per_step": statistics.mean(te), "h2d_bytes_per_step": int(w.pts.nbytes),
                      "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in hout.values())),
                      "api": "dpc_run_host"}
        # CPU oracle on a bounded sample
        v, dt, th = cpu_oracle_sample(w.pts, w.d_cut, args.cpu_sample, 99)
        res["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": th, "kind": "oracle",
                               "sample": "rho, lambda, delta of %d seeded sample points of the full %s "
                                         "(O(n) each from the definitions, labels omitted), %.1f s wall"
                                         % (min(args.cpu_sample, n), w.name, dt)}
    res["clocks"] = clocks
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = load_workload(args.workload)
    m = 512
    for s in range(args.warmup):
        cpu_oracle_sample(w.pts, w.d_cut, 64, 1000 + s)
    vals, secs = [], []
    th = 1
    for s in range(args.steps):
        v, dt, th = cpu_oracle_sample(w.pts, w.d_cut, m, 2000 + s)
        vals.append(v)
        secs.append(dt)
    value = m * len(w.d_cut) * len(secs) / sum(secs)
    ms = 1e3 * sum(secs) / len(secs)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "d_cut": w.d_cut},
            "cpu_baseline": {"kind": "oracle", "cores": th, "value": value,
                             "sample": "%d seeded sample points of %s per step (rho, lambda, delta from the "
                                       "definitions; labels omitted)" % (m, w.name)},
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
    res = run_ours(args, rank, world, dev)
    if res is not None:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
