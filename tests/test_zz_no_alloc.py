"""The allocation-free density entry point (dpc_density_static).

It serves callers that cannot let a library allocate device memory: a host
application that hands out all device memory through its own allocator or
budget, and latency-critical paths where cudaMalloc/cudaFree may synchronize
the device.  Checked here through the C ABI against the allocating
dpc_density and against the oracle, on calls back to back, exactly (the same
tolerance as every parity test: none).  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _case(kind, d, n, seed):
    if kind == "wide":
        # a box about 1e5 cutoffs wide: more fine-grid bits per axis than
        # four gridded axes can hold in a 63-bit cell code
        return W.wide_clusters(n, d, seed, extent=2.0e6, sigma=20.0)
    dtype = np.int32 if kind == "i32" else np.float32
    scale = 500.0 if dtype == np.int32 else 1.0
    return W.random_blobs(n, d, seed, dtype=dtype, scale=scale, dup_frac=0.02)


CASES = [  # different point sets, one call each, back to back
    ("f32 d=2", "f32", 2, 30000, 0.02, 11),
    ("i32 d=3", "i32", 3, 20000, 40.0, 12),
    ("i32 d=5 wide", "wide", 5, 20000, 40.0, 14),
    ("f32 d=7", "f32", 7, 12000, 0.05, 15),
]


def test_static_matches_allocating_entry_point_twice():
    for name, kind, d, n, dc, seed in CASES:
        pts = _case(kind, d, n, seed)
        want = oracle.density(pts, dc)
        assert want.max() > 1, name  # the case has neighbours to count
        t = torch.from_numpy(pts).cuda()
        for prec in ("fp32", "fp64"):
            ref = dpc.dpc_density(t, dpc.Batch.single(n, d, [dc]), precision=prec, sync=True)[0]
            for call in range(2):
                got = dpc.dpc_density_static(t, dc, precision=prec, sync=True)
                assert torch.equal(got, ref), (prec, name, call)
                assert np.array_equal(got.cpu().numpy(), want), (prec, name, call)


def test_static_limits():
    lib = dpc.load()
    p = ctypes.c_void_p(1)
    too_many = dpc.DPC_STATIC_MAX_POINTS + 1
    assert lib.dpc_density_static(p, dpc.DPC_F32, too_many, 2, 1.0, p, 1, None) == dpc.DPC_ERR_OVERFLOW
    assert lib.dpc_density_static(p, dpc.DPC_F32, 10, 9, 1.0, p, 1, None) == dpc.DPC_ERR_ARG
    # the largest size still works and matches
    n = dpc.DPC_STATIC_MAX_POINTS
    pts = W.random_blobs(n, 2, 13)
    t = torch.from_numpy(pts).cuda()
    ref = dpc.dpc_density(t, dpc.Batch.single(n, 2, [0.01]), sync=True)[0]
    got = dpc.dpc_density_static(t, 0.01, sync=True)
    assert torch.equal(got, ref)
    assert np.array_equal(got.cpu().numpy(), oracle.density(pts, 0.01))
