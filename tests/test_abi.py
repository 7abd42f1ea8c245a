"""The C ABI without a GPU: the library builds, loads, exports every entry
point that include/dpc.h declares, and rejects bad arguments on the host
before touching CUDA."""
import ctypes
import math
import os
import re

import pytest

import paper_2305_11335_gb300 as dpc
from paper_2305_11335_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return dpc.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "dpc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dpc_density", "dpc_dependent", "dpc_cluster", "dpc_run"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(dpc.EXPORTS)


def test_strerror_and_version(lib):
    assert dpc.version().count(".") == 2
    for code in range(-7, 1):
        assert dpc.strerror(code)
    assert dpc.strerror(-99) == "unknown status"


def _batch(n=10, d=2, cuts=(1.0,)):
    return dpc.Batch.single(n, d, list(cuts))


def _call_run(lib, batch, params=None, dtype=dpc.DPC_F32, flags=1, ptr=1):
    if params is None:
        params = dpc.make_params(batch if batch is not None else _batch(), 1, 1, 1.0)
    p = ctypes.c_void_p(ptr)
    return lib.dpc_run(p, dtype, batch.ptr if batch is not None else None, params, p, p, p, p, flags, None)


def test_argument_errors_are_host_side(lib):
    # every case below fails before any CUDA call, so it runs without a GPU
    assert _call_run(lib, None) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(d=9)) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(d=0)) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(cuts=(math.nan,))) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(cuts=(-1.0,))) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(cuts=(math.inf,))) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(), dtype=7) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(), flags=0xF) == dpc.DPC_ERR_UNSUPPORTED
    assert _call_run(lib, _batch(), flags=1 << 24) == dpc.DPC_ERR_ARG
    assert _call_run(lib, _batch(), ptr=0) == dpc.DPC_ERR_ARG
    b = _batch()
    assert _call_run(lib, b, params=dpc.make_params(b, 1, 1, math.nan)) == dpc.DPC_ERR_ARG
    big = dpc.Batch([0, 1 << 31], [2], [[1.0]])
    assert _call_run(lib, big) == dpc.DPC_ERR_OVERFLOW
    big_total = dpc.Batch([0, 3 << 29, 6 << 29], [2, 3], [[1.0], [1.0]])  # each < 2^31, sum >= 2^31
    assert _call_run(lib, big_total) == dpc.DPC_ERR_OVERFLOW
    bad_order = dpc.Batch([0, 5, 3], [2, 2], [[1.0], [1.0]])
    assert _call_run(lib, bad_order) == dpc.DPC_ERR_ARG
    p = ctypes.c_void_p(1)
    assert lib.dpc_dependent(p, 1, b.ptr, 1, p, 0, p, p, 1, None) == dpc.DPC_ERR_ARG  # cutoff index
    assert lib.dpc_cluster(b.ptr, 0, None, p, p, p, p, 0, None) == dpc.DPC_ERR_ARG    # no params
    skip = 1 | dpc.DPC_FLAG_SKIP_NOISE  # dpc_run only
    assert lib.dpc_density(p, 1, b.ptr, p, skip, None) == dpc.DPC_ERR_ARG
    assert lib.dpc_dependent(p, 1, b.ptr, 0, p, 0, p, p, skip, None) == dpc.DPC_ERR_ARG
    assert lib.dpc_get_stats(None, None) == dpc.DPC_ERR_ARG
    dg = lib.dpc_decision_graph
    assert dg(None, p, p, 4, p, p, 0, 0, 1.0, None, 0, None) == dpc.DPC_ERR_ARG
    assert dg(b.ptr, p, p, -1, p, p, 0, 0, 1.0, None, 0, None) == dpc.DPC_ERR_ARG     # k < 0
    assert dg(b.ptr, p, p, 1025, p, p, 0, 0, 1.0, None, 0, None) == dpc.DPC_ERR_ARG   # k > 1024
    assert dg(b.ptr, p, p, 4, None, p, 0, 0, 1.0, None, 0, None) == dpc.DPC_ERR_ARG  # no top
    assert dg(b.ptr, p, p, 0, None, None, 4, 0, 1.0, p, 0, None) == dpc.DPC_ERR_ARG  # one bin count 0
    assert dg(b.ptr, p, p, 0, None, None, 33, 4, 1.0, p, 0, None) == dpc.DPC_ERR_ARG  # rho bins > 32
    assert dg(b.ptr, p, p, 0, None, None, 4, 4, 0.0, p, 0, None) == dpc.DPC_ERR_ARG   # delta_lo 0
    assert dg(b.ptr, p, p, 0, None, None, 4, 4, math.inf, p, 0, None) == dpc.DPC_ERR_ARG
    assert dg(b.ptr, p, p, 0, None, None, 4, 4, 1.0, None, 0, None) == dpc.DPC_ERR_ARG  # no hist
    assert dg(b.ptr, None, p, 4, p, p, 0, 0, 1.0, None, 0, None) == dpc.DPC_ERR_ARG  # no rho
    assert dg(b.ptr, p, p, 4, p, p, 0, 0, 1.0, None, 1 << 10, None) == dpc.DPC_ERR_ARG  # flag
    pr = lib.dpc_priority_range
    assert pr(p, 1, None, p, 1, p, p, p, 0, p, None, 0, None) == dpc.DPC_ERR_ARG      # no batch
    assert pr(p, 7, b.ptr, p, 1, p, p, p, 0, p, None, 0, None) == dpc.DPC_ERR_ARG     # dtype
    assert pr(p, 1, b.ptr, p, -1, p, p, p, 0, p, None, 0, None) == dpc.DPC_ERR_ARG    # n_query < 0
    assert pr(p, 1, b.ptr, p, 1, p, p, p, -1, p, None, 0, None) == dpc.DPC_ERR_ARG    # max_out < 0
    assert pr(p, 1, b.ptr, p, 1, None, p, p, 0, p, None, 0, None) == dpc.DPC_ERR_ARG  # no q_inst
    assert pr(p, 1, b.ptr, p, 1, p, p, p, 4, p, None, 0, None) == dpc.DPC_ERR_ARG     # no ids
    assert pr(p, 1, b.ptr, p, 1, p, p, p, 0, None, None, 0, None) == dpc.DPC_ERR_ARG  # no count
    assert pr(p, 1, b.ptr, p, 1, p, p, p, 0, p, None, 1 << 15, None) == dpc.DPC_ERR_ARG  # flag
    assert pr(p, 1, b.ptr, p, 0, None, None, None, 0, None, None, 0, None) == dpc.DPC_OK  # no queries


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    b = _batch()
    assert _call_run(lib, b) == dpc.DPC_ERR_CUDA
