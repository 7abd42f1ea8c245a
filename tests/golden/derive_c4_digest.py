"""Compute the oracle's results for the whole batched workload (4096
instances x 8 cutoffs) and store one digest per instance.

Writes ``tests/golden/c4_oracle_digest.json``.  Run from the repository root:

    python tests/golden/derive_c4_digest.py [threads]

The full outputs (rho, lambda, delta, labels of 1.6e8 points at 8 cutoffs)
are about 25 GB and take the kd-tree oracle about half an hour on 8 cores, too
much to store or to recompute inside a test run; the GPU parity test hashes
its own outputs the same way (tests/_digest.py) and compares instance by
instance, and recomputes any instance that differs with the oracle to report
the differing elements.  The input digest guards against a generator that
draws different points on another machine.

Every number comes from ``oracle`` routines (oracle.tree_batch for rho,
lambda, delta; oracle.cluster for labels); nothing here runs the CUDA path.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from _digest import batch_input_digest, instance_digest  # noqa: E402

OUT = os.path.join(HERE, "c4_oracle_digest.json")


def oracle_instances(w, ids, nthreads=0):
    """rho, lam, delta, label of the instances ``ids`` (in that order), packed:
    (outputs [ncut][M], point offsets of each listed instance)."""
    parts = [w.instance(int(i)).reshape(-1) for i in ids]
    flat = np.concatenate(parts) if parts else np.zeros(0, np.float32)
    po = np.concatenate([[0], np.cumsum([w.sizes[int(i)] for i in ids])]).astype(np.int64)
    co = np.concatenate([[0], np.cumsum([p.size for p in parts])[:-1]]).astype(np.int64)
    dims = [w.dims[int(i)] for i in ids]
    cuts = [w.d_cut[int(i)] for i in ids]
    r = oracle.tree_batch(flat, po, co, dims, cuts, nthreads=nthreads)
    ncut = len(cuts[0])
    label = np.zeros_like(r["rho"])
    for t, i in enumerate(ids):
        lo, hi = po[t], po[t + 1]
        for c in range(ncut):
            j = int(i) * ncut + c
            label[c, lo:hi] = oracle.cluster(r["rho"][c, lo:hi], r["lam"][c, lo:hi], r["delta"][c, lo:hi],
                                             w.rho_noise[j], w.rho_min[j], w.delta_min[j])
    r["label"] = label
    return r, po


def main():
    nthreads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    t0 = time.time()
    w = W.c4()
    digests = [None] * w.n_inst
    group = 256
    for g0 in range(0, w.n_inst, group):
        ids = list(range(g0, min(w.n_inst, g0 + group)))
        r, po = oracle_instances(w, ids, nthreads)
        for t, i in enumerate(ids):
            digests[i] = instance_digest(r["rho"], r["lam"], r["delta"], r["label"], po[t], po[t + 1])
        print("instances %d..%d done, %.0f s" % (ids[0], ids[-1], time.time() - t0), flush=True)
    out = {"what": "per-instance sha256 prefixes (tests/_digest.py) of the oracle's rho, lambda, delta "
                   "and labels for the 4096-instance batched workload at its 8 cutoffs",
           "workload": w.name, "input_sha256": batch_input_digest(w), "instances": digests,
           "oracle": "oracle.tree_batch + oracle.cluster", "seconds": round(time.time() - t0, 1),
           "threads": oracle.threads(nthreads)}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
