"""The allocation-free density entry point (dpc_density_static).

It serves callers that cannot let a library allocate device memory (stream
capture into a CUDA graph, externally budgeted device memory, paths that
cannot afford an allocation's synchronization).  Checked here through the C
ABI against the allocating dpc_density on two calls in a row, exactly (the
same tolerance as every parity test: none).  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2305_11335_gb300 as dpc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


CASES = [  # two different point sets, one call each, back to back
    ("f32 d=2", np.float32, 2, 30000, 0.02, 11),
    ("i32 d=3", np.int32, 3, 20000, 40.0, 12),
]


def test_static_matches_allocating_entry_point_twice():
    for prec in ("fp32", "fp64"):
        for name, dtype, d, n, dc, seed in CASES:
            scale = 500.0 if dtype == np.int32 else 1.0
            pts = W.random_blobs(n, d, seed, dtype=dtype, scale=scale, dup_frac=0.02)
            t = torch.from_numpy(pts).cuda()
            ref = dpc.dpc_density(t, dpc.Batch.single(n, d, [dc]), precision=prec, sync=True)[0]
            got = dpc.dpc_density_static(t, dc, precision=prec, sync=True)
            assert torch.equal(got, ref), (prec, name)


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
