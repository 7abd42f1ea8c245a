"""Helpers for the GPU parity tests: run the CUDA library through the C ABI
and compare with the CPU oracle element by element.

Tolerance: none.  rho, lambda and labels are integers and must be equal;
delta must be bit-identical binary64 (the library re-evaluates every
candidate that could decide the winner with the canonical binary64 distance,
and delta is sqrt of that distance, correctly rounded on both sides).
"""
import numpy as np
import torch

import oracle
import paper_2305_11335_gb300 as dpc


def gpu_run(pts, d_cuts, rho_noise, rho_min, delta_min, precision="fp32"):
    t = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    out = dpc.run(t, list(d_cuts), rho_noise, rho_min, delta_min, precision=precision, sync=True)
    return {k: v.cpu().numpy() for k, v in out.items()}


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def assert_same(got, ref, what=""):
    for k in ("rho", "lam", "label"):
        if not np.array_equal(got[k], ref[k]):
            bad = np.flatnonzero(got[k] != ref[k])
            raise AssertionError("%s %s differs at %d ids, first %s: got %s want %s" % (
                what, k, len(bad), bad[:5].tolist(), got[k][bad[:5]].tolist(), ref[k][bad[:5]].tolist()))
    if not np.array_equal(bits(got["delta"]), bits(ref["delta"])):
        bad = np.flatnonzero(bits(got["delta"]) != bits(ref["delta"]))
        raise AssertionError("%s delta differs at %d ids, first %s: got %r want %r" % (
            what, len(bad), bad[:5].tolist(), got["delta"][bad[:5]].tolist(), ref["delta"][bad[:5]].tolist()))


def parity(pts, d_cuts, rho_noise=2, rho_min=3, delta_min=1.0, precisions=("fp32", "fp64")):
    """Full-array parity for every cutoff and both precision modes."""
    d_cuts = list(d_cuts) if isinstance(d_cuts, (list, tuple)) else [d_cuts]
    refs = [oracle.run(pts, dc, rho_noise, rho_min, delta_min) for dc in d_cuts]
    for prec in precisions:
        got = gpu_run(pts, d_cuts, rho_noise, rho_min, delta_min, prec)
        for c, ref in enumerate(refs):
            assert_same({k: v[c] for k, v in got.items()}, ref, "%s cut=%r" % (prec, d_cuts[c]))
    return refs
