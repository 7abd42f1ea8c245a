"""Batched calls (many instances of mixed dimension, each with its own cutoff
sweep and thresholds) against the oracle, instance by instance.

A batch runs as classes of equal padded dimension, every kernel launched once
per class; these tests put many instances in every class, including empty,
single-point and ragged (non-multiple-of-32) instances, and check every
output element of every instance and cutoff, bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W
from _gpu_util import assert_same

pytestmark = pytest.mark.gpu

NCUT = 3


def make_batch(seed, n_inst, dims, dtype=np.float32, max_n=2500):
    rng = np.random.default_rng(seed)
    sizes, insts, cuts = [], [], []
    special = [0, 1, 2, 31, 32, 33, 64, 65]
    for i in range(n_inst):
        d = int(dims[i % len(dims)])
        n = special[i] if i < len(special) else int(rng.integers(3, max_n))
        if dtype == np.int32:
            p = rng.integers(0, 60, (n, d)).astype(np.int32)
            base = [1.0, 2.0, 3.5]
        else:
            p = W.random_blobs(n, d, 1000 + seed * 100 + i) if n else np.zeros((0, d), np.float32)
            base = [0.03 * (1 + 0.4 * (d - 1)) * f for f in (1.0, 1.25, 1.5625)]
        sizes.append(n)
        insts.append(p)
        cuts.append(base)
    return sizes, [int(dims[i % len(dims)]) for i in range(n_inst)], insts, cuts


def thresholds(n_inst, seed):
    rng = np.random.default_rng(seed)
    rn = rng.integers(1, 4, n_inst * NCUT).tolist()
    rm = [r + int(x) for r, x in zip(rn, rng.integers(0, 5, n_inst * NCUT))]
    dm = rng.uniform(0.02, 0.3, n_inst * NCUT).tolist()
    return rn, rm, dm


def check_run(sizes, dims, insts, cuts, dtype, precision, seed, layout="auto", skip_noise=False, graph=False):
    batch = dpc.Batch.packed(sizes, dims, cuts)
    flat = np.concatenate([p.reshape(-1) for p in insts]).astype(dtype)
    t = torch.from_numpy(flat).cuda()
    rn, rm, dm = thresholds(len(sizes), seed)
    params = dpc.make_params(batch, rn, rm, dm)
    if graph:
        with torch.cuda.stream(torch.cuda.Stream()):
            for _ in range(2):
                out = dpc.dpc_run(t, batch, params, precision=precision, sync=True, layout=layout,
                                  skip_noise=skip_noise, graph=True)
    else:
        out = dpc.dpc_run(t, batch, params, precision=precision, sync=True, layout=layout, skip_noise=skip_noise)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    for i, p in enumerate(insts):
        lo, hi = batch.pt_offset[i], batch.pt_offset[i + 1]
        for c in range(NCUT):
            j = i * NCUT + c
            ref = oracle.run(p, cuts[i][c], rn[j], rm[j], dm[j], rho_skip=rn[j] if skip_noise else 0)
            assert_same({k: v[c, lo:hi] for k, v in out.items()}, ref,
                        "%s inst %d (n=%d d=%d) cut %d" % (precision, i, sizes[i], dims[i], c))


@pytest.mark.parametrize("precision,layout", [("fp32", "auto"), ("fp64", "auto"), ("fp32", "union"),
                                              ("fp32", "segment"), ("fp64", "segment"), ("fp32", "tree"),
                                              ("fp64", "tree"), ("fp32", "tensor"), ("fp64", "tensor"),
                                              ("fp32", "pairs"), ("fp64", "pairs"), ("fp32", "cell"),
                                              ("fp64", "cell")])
def test_batch_mixed_dims_float(precision, layout):
    sizes, dims, insts, cuts = make_batch(1, 48, [2, 3, 5, 1, 4, 7, 8, 2, 3, 5])
    check_run(sizes, dims, insts, cuts, np.float32, precision, 11, layout)


@pytest.mark.parametrize("layout", ["union", "segment", "tree", "tensor", "pairs", "cell"])
def test_batch_int_ties(layout):
    sizes, dims, insts, cuts = make_batch(2, 30, [2, 3], dtype=np.int32, max_n=1500)
    check_run(sizes, dims, insts, cuts, np.int32, "fp32", 12, layout)


def test_batch_one_class_many_instances():
    """300 small 2-D instances: one class, the instance field of the sort key
    9 bits wide."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(1, 200, 300)]
    insts = [W.random_blobs(n, 2, 5000 + i) for i, n in enumerate(sizes)]
    dims = [2] * len(sizes)
    cuts = [[0.03, 0.04, 0.05] for _ in sizes]
    check_run(sizes, dims, insts, cuts, np.float32, "fp32", 13)


@pytest.mark.parametrize("layout,graph", [("auto", False), ("tree", False), ("segment", False), ("cell", False),
                                          ("auto", True)])
def test_batch_skip_noise(layout, graph):
    """Noise points skip the dependent search (lambda -1, delta NaN); every
    instance and cutoff has its own noise threshold."""
    sizes, dims, insts, cuts = make_batch(21, 30, [1, 2, 3, 4, 6])
    check_run(sizes, dims, insts, cuts, np.float32, "fp32", 22, layout=layout, skip_noise=True, graph=graph)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_skip_noise(precision):
    pts = W.random_blobs(20000, 2, 77)
    cuts = [0.01, 0.02]
    t = torch.from_numpy(pts).cuda()
    out = dpc.run(t, cuts, 4, 6, 0.05, precision=precision, skip_noise=True)
    for c, dc in enumerate(cuts):
        ref = oracle.run(pts, dc, 4, 6, 0.05, rho_skip=4)
        assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref, "cut %d" % c)
        assert np.isnan(ref["delta"]).sum() == (ref["rho"] < 4).sum() > 0


def test_batch_split_entry_points():
    sizes, dims, insts, cuts = make_batch(3, 24, [2, 3, 5])
    batch = dpc.Batch.packed(sizes, dims, cuts)
    t = torch.from_numpy(np.concatenate([p.reshape(-1) for p in insts]).astype(np.float32)).cuda()
    rn, rm, dm = thresholds(len(sizes), 14)
    params = dpc.make_params(batch, rn, rm, dm)
    rho = dpc.dpc_density(t, batch, sync=True)
    c = 1
    lam, delta = dpc.dpc_dependent(t, batch, c, rho[c].contiguous(), sync=True)
    label = dpc.dpc_cluster(batch, c, params, rho[c].contiguous(), lam, delta, sync=True)
    got = {"rho": rho[c].cpu().numpy(), "lam": lam.cpu().numpy(), "delta": delta.cpu().numpy(),
           "label": label.cpu().numpy()}
    for i, p in enumerate(insts):
        lo, hi = batch.pt_offset[i], batch.pt_offset[i + 1]
        j = i * NCUT + c
        ref = oracle.run(p, cuts[i][c], rn[j], rm[j], dm[j])
        assert_same({k: v[lo:hi] for k, v in got.items()}, ref, "inst %d" % i)
        for cc in range(NCUT):
            assert np.array_equal(rho[cc].cpu().numpy()[lo:hi], oracle.density(p, cuts[i][cc]))


def test_batch_coord_offsets_out_of_order():
    """Coordinates stored in reverse instance order with gaps between them."""
    sizes, dims, insts, cuts = make_batch(4, 12, [2, 5, 3])
    co, parts, pos = [0] * len(sizes), [np.full(7, -1e30, np.float32)], 7
    for i in reversed(range(len(sizes))):
        co[i] = pos
        parts.append(insts[i].reshape(-1).astype(np.float32))
        parts.append(np.full(5, -1e30, np.float32))
        pos += insts[i].size + 5
    flat = np.concatenate(parts)
    po = [0]
    for n in sizes:
        po.append(po[-1] + n)
    batch = dpc.Batch(po, dims, cuts, coord_offset=co)
    rn, rm, dm = thresholds(len(sizes), 15)
    params = dpc.make_params(batch, rn, rm, dm)
    out = dpc.dpc_run(torch.from_numpy(flat).cuda(), batch, params, sync=True)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    for i, p in enumerate(insts):
        lo, hi = po[i], po[i + 1]
        assert np.array_equal(flat[co[i]:co[i] + p.size], p.reshape(-1))
        for c in range(NCUT):
            j = i * NCUT + c
            ref = oracle.run(p, cuts[i][c], rn[j], rm[j], dm[j])
            assert_same({k: v[c, lo:hi] for k, v in out.items()}, ref, "inst %d cut %d" % (i, c))
