"""Priority range search against the oracle, query by query: every count and
every returned id exact.

Queries: random boxes from a point's neighbourhood up to the whole domain,
degenerate boxes (one point), empty boxes (lo > hi), a NaN bound, thresholds
below every priority and above every priority; batches of mixed dimension
with empty, single-point and ragged instances; int32 and float32 points;
outputs truncated to fewer ids than matches; and the per-lane walk that takes
over when a warp's node stack is full.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W

pytestmark = pytest.mark.gpu


def make_queries(rng, insts, rhos, nq):
    q_inst, lo, hi, rq = [], [], [], []
    nonempty = [i for i, p in enumerate(insts) if len(p)]
    for k in range(nq):
        i = int(rng.choice(nonempty))
        p = insts[i].astype(np.float64)
        d = p.shape[1]
        c = p[int(rng.integers(0, len(p)))]
        span = p.max(axis=0) - p.min(axis=0) + 1.0
        kind = k % 8
        if kind == 0:    # the whole instance
            a, b = p.min(axis=0), p.max(axis=0)
        elif kind == 1:  # one point exactly
            a, b = c.copy(), c.copy()
        elif kind == 2:  # empty: lo > hi on one axis
            a, b = c - 0.1 * span, c + 0.1 * span
            a[0], b[0] = c[0] + 1.0, c[0] - 1.0
        else:            # a box around a point, random size per axis
            w = span * 10.0 ** rng.uniform(-3, -0.3, d)
            a, b = c - w * rng.random(d), c + w * rng.random(d)
        t = int(rng.choice([-1, 0, int(np.median(rhos[i])) if len(rhos[i]) else 0,
                            int(rhos[i].max()) if len(rhos[i]) else 0, 1 << 30]))
        q_inst.append(i)
        lo.append(np.pad(a, (0, 8 - d)))
        hi.append(np.pad(b, (0, 8 - d)))
        rq.append(t)
    return q_inst, np.array(lo), np.array(hi), rq


def check(insts, dims, rhos, nq, max_out, seed, dtype=np.float32, nan_query=False):
    rng = np.random.default_rng(seed)
    sizes = [len(p) for p in insts]
    batch = dpc.Batch.packed(sizes, dims, [[1.0]] * len(sizes))
    flat = np.concatenate([p.reshape(-1) for p in insts]).astype(dtype)
    rho = np.concatenate(rhos).astype(np.int32)
    q_inst, lo, hi, rq = make_queries(rng, insts, rhos, nq)
    if nan_query:
        lo[0, 0] = math.nan
    box = dpc.range_boxes(lo, hi)
    out = dpc.dpc_priority_range(torch.from_numpy(flat).cuda(), batch, torch.from_numpy(rho).cuda(),
                                 torch.tensor(q_inst, dtype=torch.int32).cuda(), box,
                                 torch.tensor(rq, dtype=torch.int32).cuda(), max_out=max_out, sync=True)
    count = out["count"].cpu().numpy()
    ids = out["ids"].cpu().numpy() if max_out else None
    for k in range(nq):
        i = q_inst[k]
        d = dims[i]
        want = oracle.priority_range(insts[i].astype(dtype), rhos[i], lo[k, :d], hi[k, :d], rq[k])
        assert count[k] == len(want), (k, i, count[k], len(want))
        if max_out:
            row = np.full(max_out, -1, np.int32)
            m = min(max_out, len(want))
            row[:m] = want[:m]
            assert np.array_equal(ids[k], row), (k, ids[k][:8], row[:8])
    return count


@pytest.mark.parametrize("max_out", [0, 5, 4096])
def test_range_single_instance(max_out):
    pts = W.random_blobs(30000, 2, 31)
    rho = oracle.density(pts, 0.02)
    count = check([pts], [2], [rho], 200, max_out, 1)
    assert (count > 0).sum() > 50


def test_range_random_priorities_with_ties_3d():
    rng = np.random.default_rng(8)
    pts = W.random_blobs(20000, 3, 32)
    check([pts], [3], [rng.integers(0, 6, 20000).astype(np.int32)], 160, 300, 2, nan_query=True)


@pytest.mark.parametrize("dtype", [np.float32, np.int32])
def test_range_batch_mixed_dims(dtype):
    rng = np.random.default_rng(9)
    sizes = [0, 1, 2, 33, 700, 5000, 1, 64, 3000, 12000]
    dims = [1, 2, 3, 5, 8, 2, 4, 7, 6, 3]
    insts, rhos = [], []
    for i, (n, d) in enumerate(zip(sizes, dims)):
        if dtype == np.int32:
            p = rng.integers(-2000, 2000, (n, d)).astype(np.int32)
        else:
            p = W.random_blobs(n, d, 600 + i) if n else np.zeros((0, d), np.float32)
        insts.append(p)
        rhos.append(rng.integers(1, 40, n).astype(np.int32))
    check(insts, dims, rhos, 400, 64, 3, dtype=dtype)


def test_range_per_lane_walk(monkeypatch):
    """A stack of 4 entries per warp sends almost every subtree to the
    per-lane walk over parent links."""
    monkeypatch.setenv("DPC_RANGE_STACK", "4")
    pts = W.random_blobs(40000, 2, 33)
    rng = np.random.default_rng(10)
    check([pts], [2], [rng.integers(0, 100, 40000).astype(np.int32)], 120, 2000, 4)


def test_range_bad_instance_is_a_data_error():
    pts = W.random_blobs(100, 2, 34)
    batch = dpc.Batch.single(100, 2, [0.1])
    box = dpc.range_boxes(np.zeros((2, 2)), np.ones((2, 2)))
    with pytest.raises(dpc.DpcError) as e:
        dpc.dpc_priority_range(torch.from_numpy(pts).cuda(), batch, torch.ones(100, dtype=torch.int32).cuda(),
                               torch.tensor([0, 1], dtype=torch.int32).cuda(), box,
                               torch.tensor([0, 0], dtype=torch.int32).cuda(), max_out=4, sync=True)
    assert e.value.code == dpc.DPC_ERR_DATA
