"""Failure detection on the GPU without a fault.

Every wait inside a kernel has an iteration limit; when it runs out the
kernel records DPC_ERR_TIMEOUT in the call's status word and finishes without
hanging or touching memory it does not own.  The environment variable
DPC_TEST_WAIT_LIMIT lowers that limit (0: every bounded wait gives up at its
first poll), so these tests make the waits run out on purpose and check
  * the call reports DPC_ERR_TIMEOUT (DPC_FLAG_SYNC_CHECK),
  * the context stays usable and the next normal call is exact against the
    oracle.
The radix sort's look-back recounts the digits of earlier tiles itself when
it gives up, so even the timed-out call's result is exact there; the
tensor-core density leaves its pieces at density 0 and only the status tells.

DPC_WORKSPACE_LIMIT_BYTES caps a single device allocation: a call that needs
a larger workspace fails with DPC_ERR_OOM on the host, before any work is
queued, and the call after the cap is lifted works.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W
from _gpu_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


class env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update({k: str(v) for k, v in self.kv.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _run(pts, d_cut, layout="auto", stream=None):
    batch = dpc.Batch.single(pts.shape[0], pts.shape[1], [d_cut])
    params = dpc.make_params(batch, 2, 3, 0.1)
    out = dpc.dpc_run(torch.from_numpy(pts).cuda(), batch, params, sync=True, layout=layout, stream=stream)
    return {k: v[0].cpu().numpy() for k, v in out.items()}


def test_sort_lookback_timeout_is_reported_and_recovers():
    pts = W.random_blobs(60000, 2, 31, dup_frac=0.01)  # 15 sort tiles: 14 look-backs per pass
    d_cut = 0.01
    ref = oracle.run(pts, d_cut, 2, 3, 0.1)
    with env(DPC_TEST_WAIT_LIMIT=0):
        with pytest.raises(dpc.DpcError) as e:
            _run(pts, d_cut)
        assert e.value.code == dpc.DPC_ERR_TIMEOUT
    assert dpc.dpc_last_status() == dpc.DPC_ERR_TIMEOUT
    got = _run(pts, d_cut)
    assert_same(got, ref, "after a timed-out call")


def test_sort_lookback_fallback_is_exact():
    """The look-back that gave up counts the earlier tiles' digits itself, so
    the timed-out call still sorts correctly and every output is exact."""
    pts = W.random_blobs(30000, 3, 32, dtype=np.int32, scale=400.0, dup_frac=0.02)
    d_cut = 12.0
    ref = oracle.run(pts, d_cut, 2, 3, 0.1)
    batch = dpc.Batch.single(pts.shape[0], 3, [d_cut])
    params = dpc.make_params(batch, 2, 3, 0.1)
    t = torch.from_numpy(pts).cuda()
    with env(DPC_TEST_WAIT_LIMIT=0):
        out = dpc.dpc_run(t, batch, params, sync=False)
        assert dpc.dpc_last_status() == dpc.DPC_ERR_TIMEOUT
    assert_same({k: v[0].cpu().numpy() for k, v in out.items()}, ref, "timed-out call")


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    pts = W.random_blobs(3000, 7, 33, dup_frac=0.01)  # one sort tile: only the MMA waits give up
    d_cut = 0.08
    ref = oracle.run(pts, d_cut, 2, 3, 0.1)
    with env(DPC_TEST_WAIT_LIMIT=0):
        with pytest.raises(dpc.DpcError) as e:
            _run(pts, d_cut, layout="tensor")
        assert e.value.code == dpc.DPC_ERR_TIMEOUT
    got = _run(pts, d_cut, layout="tensor")
    assert_same(got, ref, "tensor layout after a timed-out call")
    assert dpc.dpc_get_stats()["density_layout"] == 4


def test_workspace_cap_gives_oom_then_recovers():
    pts = W.random_blobs(20000, 2, 34)
    d_cut = 0.01
    ref = oracle.run(pts, d_cut, 2, 3, 0.1)
    s = torch.cuda.Stream()  # a stream of its own: its workspace does not exist yet
    with env(DPC_WORKSPACE_LIMIT_BYTES=4096):
        with pytest.raises(dpc.DpcError) as e:
            _run(pts, d_cut, stream=s)
        assert e.value.code == dpc.DPC_ERR_OOM
    got = _run(pts, d_cut, stream=s)
    assert_same(got, ref, "after the cap is lifted")
