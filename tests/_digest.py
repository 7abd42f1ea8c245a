"""Digests of DPC outputs and inputs, so that results the oracle computed
once can be compared with a later run without storing the arrays.

Only hashing lives here (no clustering arithmetic): the same byte layout is
hashed on both sides, instance by instance.
"""
import hashlib

import numpy as np


def instance_digest(rho, lam, delta, label, lo, hi):
    """sha256 prefix of one instance's outputs: for every cutoff row c, the
    bytes of rho[c, lo:hi] (int32), lam (int32), delta (float64) and label
    (int32), little-endian, in that order."""
    h = hashlib.sha256()
    for c in range(rho.shape[0]):
        for a, dt in ((rho, "<i4"), (lam, "<i4"), (delta, "<f8"), (label, "<i4")):
            h.update(np.ascontiguousarray(a[c, lo:hi], dtype=dt).tobytes())
    return h.hexdigest()[:16]


def batch_input_digest(w):
    """sha256 of a batched workload's inputs: coordinates, sizes, dimensions,
    cutoffs and thresholds."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(w.flat, dtype="<f4").tobytes())
    for a, dt in ((w.sizes, "<i8"), (w.dims, "<i4"), (w.coord_offset, "<i8"), (w.d_cut, "<f8"),
                  (w.rho_noise, "<i8"), (w.rho_min, "<i8"), (w.delta_min, "<f8")):
        h.update(np.ascontiguousarray(np.asarray(a), dtype=dt).tobytes())
    return h.hexdigest()
