"""Derive the data-dependent workload parameters with the CPU oracle alone.

Writes ``tests/golden/workload_params.json``.  Run from the repository root:

    python tests/golden/derive_workload_params.py

Rules (the paper leaves d_cut to the user, Section 3; its synthetic sets use a
fixed d_cut = 30, Table 2):

* c2: d_cut = the median, over 4096 seeded sample points, of the distance to
  the 30th nearest point (the point itself counted first), so the median
  density is about 30.  rho_noise = rho_min = 2 x the median density of 1024
  seeded sample points at that d_cut.
* c3: d_cut = 30 (given).  rho_noise = rho_min = 2 x median density (1024
  sample points).
* c5: d_cut0 from the same 30th-nearest rule (2048 sample points); the sweep is
  d_cut0 * 1.25^k, k = 0..3, with rho_min = 2 x median density at each cutoff
  (1024 sample points).
* c4 (``--c4``, written to ``tests/golden/c4_params.json``): per instance,
  d_cut0 = the median distance to the 8th nearest point (self counted first)
  over 1024 seeded sample points; rho_min = 2 x median density over 256
  seeded sample points at each cutoff d_cut0 * 1.25^k, k = 0..7.

Every number comes from ``oracle`` routines; nothing here runs the CUDA path.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_params.json")
OUT_C4 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_params.json")


def sample(n, m, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(m, n), replace=False)).astype(np.int64)


def median_rho(pts, d_cut, seed, m=1024):
    idx = sample(pts.shape[0], m, seed)
    return float(np.median(oracle.density(pts, d_cut, idx=idx)))


def kth_cut(pts, k, m, seed):
    idx = sample(pts.shape[0], m, seed)
    s = oracle.kth_sqdist(pts, idx, k)
    return float(np.sqrt(np.median(s)))


def main():
    out = {}
    t = time.time()
    pts, _ = W.c2_points()
    dc = kth_cut(pts, 30, 4096, 102)
    med = median_rho(pts, dc, 202)
    out["c2"] = {"d_cut": dc, "median_rho_sample": med, "rho_min": int(round(2 * med))}
    print("c2", out["c2"], "%.1fs" % (time.time() - t), flush=True)

    t = time.time()
    pts, _ = W.c5_points()
    dc0 = kth_cut(pts, 30, 2048, 105)
    meds = [median_rho(pts, dc0 * 1.25 ** k, 205 + k) for k in range(4)]
    out["c5"] = {"d_cut0": dc0, "median_rho_sample": meds, "rho_min": [int(round(2 * m)) for m in meds]}
    print("c5", out["c5"], "%.1fs" % (time.time() - t), flush=True)

    t = time.time()
    pts, _ = W.c3_points()
    med = median_rho(pts, 30.0, 203)
    out["c3"] = {"d_cut": 30.0, "median_rho_sample": med, "rho_min": int(round(2 * med))}
    print("c3", out["c3"], "%.1fs" % (time.time() - t), flush=True)

    out["_how"] = "tests/golden/derive_workload_params.py (CPU oracle only)"
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


def main_c4():
    t = time.time()
    specs = W.c4_instance_specs()
    d0, rmins = [], []
    for i, s in enumerate(specs):
        pts = W.c4_instance(s)
        dc = kth_cut(pts, 8, 1024, 10_000 + i)
        d0.append(dc)
        rmins.append([int(round(2 * median_rho(pts, dc * 1.25 ** k, 20_000 + 8 * i + k, m=256)))
                      for k in range(W.C4_NCUT)])
        if i % 512 == 0:
            print("c4", i, dc, rmins[-1], "%.1fs" % (time.time() - t), flush=True)
    with open(OUT_C4, "w") as f:
        json.dump({"_how": "tests/golden/derive_workload_params.py --c4 (CPU oracle only)",
                   "d_cut0": d0, "rho_min": rmins}, f, separators=(",", ":"))
        f.write("\n")
    print("c4 done %.1fs" % (time.time() - t))


if __name__ == "__main__":
    if "--c4" in sys.argv:
        main_c4()
    else:
        main()
