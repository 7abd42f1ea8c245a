"""Decision-graph summaries (top-k by gamma = rho * delta, log2-binned
(rho, delta) counts) against the oracle, instance by instance, bit for bit.

Inputs are seeded synthetic (rho, delta) arrays with the structure the
pipeline produces -- small integer densities with many exact ties, one +inf
delta per instance, NaN deltas of skipped points -- and, in one test, the
oracle's own rho and delta of clustered point sets.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W
from _gpu_util import bits

pytestmark = pytest.mark.gpu


def synthetic(n, seed, ties=True):
    rng = np.random.default_rng(seed)
    if ties:
        rho = rng.integers(1, 9, n).astype(np.int32)
        delta = rng.choice(np.array([0.0, 0.01, 0.02, 0.5, 1.0, 3.0, 1e-9, 7e5]), n)
    else:
        rho = rng.integers(1, 1 << 24, n).astype(np.int32)
        delta = rng.random(n) * 10.0 ** rng.integers(-6, 6, n)
    if n:
        delta[rng.integers(0, n, max(1, n // 50))] = math.nan
        delta[int(rng.integers(0, n))] = math.inf
    return rho, delta


def check(sizes, arrays, k, rho_bins, delta_bins, delta_lo):
    dims = [2] * len(sizes)
    batch = dpc.Batch.packed(sizes, dims, [[1.0]] * len(sizes))
    rho = np.concatenate([a[0] for a in arrays]).astype(np.int32) if sizes else np.zeros(0, np.int32)
    delta = np.concatenate([a[1] for a in arrays]).astype(np.float64)
    out = dpc.dpc_decision_graph(batch, torch.from_numpy(rho).cuda(), torch.from_numpy(delta).cuda(), k=k,
                                 rho_bins=rho_bins, delta_bins=delta_bins, delta_lo=delta_lo, sync=True)
    out = {key: v.cpu().numpy() for key, v in out.items()}
    for i, (r, d) in enumerate(arrays):
        ref = oracle.decision_graph(r, d, k, rho_bins, delta_bins, delta_lo)
        if k:
            assert np.array_equal(out["top"][i], ref["top"]), (i, sizes[i], out["top"][i][:8], ref["top"][:8])
            assert np.array_equal(bits(out["gamma"][i]), bits(ref["gamma"])), i
        if rho_bins:
            assert np.array_equal(out["hist"][i], ref["hist"]), i


@pytest.mark.parametrize("k", [1, 5, 64, 1024])
def test_decision_graph_ties_ragged_batch(k):
    sizes = [0, 1, 2, 31, 33, 1000, 0, 5000, 70000]
    arrays = [synthetic(n, 40 + i) for i, n in enumerate(sizes)]
    check(sizes, arrays, k, 16, 40, 0.01)


def test_decision_graph_distinct_values():
    sizes = [4097, 300000]
    arrays = [synthetic(n, 70 + i, ties=False) for i, n in enumerate(sizes)]
    check(sizes, arrays, 1024, 32, 64, 1e-6)


def test_decision_graph_all_equal_and_all_skipped():
    n = 3000
    eq = (np.full(n, 4, np.int32), np.full(n, 0.25))   # every gamma 1.0: the smallest ids win
    skip = (np.ones(n, np.int32), np.full(n, math.nan))  # no point takes part
    check([n, n], [eq, skip], 100, 4, 4, 0.5)


def test_decision_graph_of_clustered_points():
    sizes, arrays = [], []
    for i, (n, d) in enumerate([(3000, 2), (2000, 3), (1500, 5)]):
        pts = W.random_blobs(n, d, 500 + i)
        ref = oracle.run(pts, 0.03 * (1 + 0.4 * (d - 1)), 2, 3, 0.1, rho_skip=2)
        sizes.append(n)
        arrays.append((ref["rho"], ref["delta"]))
    check(sizes, arrays, 32, 12, 24, 1e-3)


def test_decision_graph_many_bins():
    """More (rho, delta) bins than fit in shared memory: counted with global
    atomics only."""
    sizes = [40000, 3000]
    arrays = [synthetic(n, 110 + i, ties=False) for i, n in enumerate(sizes)]
    check(sizes, arrays, 0, 32, 200, 1e-7)


def test_decision_graph_products_only_one_kind():
    sizes = [500, 800]
    arrays = [synthetic(n, 90 + i) for i, n in enumerate(sizes)]
    check(sizes, arrays, 0, 8, 8, 0.1)   # histogram only
    check(sizes, arrays, 7, 0, 0, 1.0)   # top-k only
