"""Python binding of the GB300 exact Density Peaks Clustering library.

A thin ctypes layer over ``libdpc.so`` (declared in ``include/dpc.h``): it
only marshals arguments.  Every step of the computation runs in the library's
CUDA kernels; PyTorch provides device memory and the current stream.  There is
no CPU fallback: if the library is not built, or no CUDA device is present,
every compute call raises.

The functions carry the C names:

* ``dpc_density(pts, batch, ...)``            -> rho      [n_dcut, N] int32
* ``dpc_dependent(pts, batch, k, rho, ...)``  -> (lambda [N] int32, delta [N] float64)
* ``dpc_cluster(batch, k, params, rho, lambda, delta)`` -> label [N] int32
* ``dpc_run(pts, batch, params, ...)``        -> dict of [n_dcut, N] tensors
* ``dpc_run_host(pts_host, batch, params, ...)`` -> dict of host tensors

``Batch.single(n, d, d_cut)`` describes one point set; ``Batch.packed`` a batch.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpc.so")

DPC_OK = 0
DPC_ERR_ARG = -1
DPC_ERR_CUDA = -2
DPC_ERR_OOM = -3
DPC_ERR_TIMEOUT = -4
DPC_ERR_OVERFLOW = -5
DPC_ERR_UNSUPPORTED = -6
DPC_ERR_DATA = -7

DPC_I32 = 0
DPC_F32 = 1
PREC = {"fp64": 0, "fp32": 1}
DPC_FLAG_SYNC_CHECK = 1 << 8

EXPORTS = ["dpc_density", "dpc_dependent", "dpc_cluster", "dpc_decision_graph", "dpc_priority_range", "dpc_run",
           "dpc_run_host", "dpc_density_static",
           "dpc_get_stats", "dpc_get_phase_times", "dpc_last_status", "dpc_strerror", "dpc_version",
           "dpc_release", "dpc_cut_band", "dpc_probe_peak"]
DPC_STATIC_MAX_POINTS = 65536


class DpcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))
        self.code = code


class _Batch(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int32), ("pt_offset", ctypes.POINTER(ctypes.c_int64)),
                ("coord_offset", ctypes.POINTER(ctypes.c_int64)), ("dim", ctypes.POINTER(ctypes.c_int32)),
                ("n_dcut", ctypes.c_int32), ("d_cut", ctypes.POINTER(ctypes.c_double))]


class _Params(ctypes.Structure):
    _fields_ = [("rho_noise", ctypes.c_int32), ("rho_min", ctypes.c_int32), ("delta_min", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("band_pairs", ctypes.c_int64), ("far_queries", ctypes.c_int64),
                ("exact_rescans", ctypes.c_int64), ("occupied_cells", ctypes.c_int64),
                ("grid_level", ctypes.c_int32), ("bits_per_axis", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("far_nodes", ctypes.c_int64),
                ("far_nodes_max", ctypes.c_int64), ("block_radius", ctypes.c_int32),
                ("density_layout", ctypes.c_int32), ("near_layout", ctypes.c_int32),
                ("near_shift", ctypes.c_int32), ("density_pairs", ctypes.c_int64)]


PHASES = ["bin", "tree", "cells", "density", "maxkey", "near", "far", "labels"]
DPC_FLAG_PHASE_TIMES = 1 << 9
DPC_FLAG_AUTOTUNE = 1 << 10
DPC_FLAG_GRAPH = 1 << 11
DPC_FLAG_SKIP_NOISE = 1 << 15


def DPC_FLAG_NEAR_SHIFT(j: int) -> int:
    """Near-dependent phase j = 0..2 grid levels below the density's; -1 = auto."""
    if j < 0:
        return 0
    if j > 2:
        raise ValueError("near shift must be 0..2")
    return (j + 1) << 20


def DPC_FLAG_RADIUS(r: int) -> int:
    return (int(r) & 7) << 12


LAYOUTS = {"auto": 0, "union": 1, "segment": 2, "tree": 3, "tensor": 4, "pairs": 5, "cell": 6}


def DPC_FLAG_LAYOUT(layout: str) -> int:
    return LAYOUTS[layout] << 16


class _PhaseTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(PHASES)), ("launches", ctypes.c_int64 * len(PHASES))]


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libdpc.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdpc.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"`" % path)
    lib = ctypes.CDLL(path)
    vp, i32, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    bp = ctypes.POINTER(_Batch)
    pp = ctypes.POINTER(_Params)
    lib.dpc_density.argtypes = [vp, ctypes.c_int, bp, vp, u32, vp]
    lib.dpc_dependent.argtypes = [vp, ctypes.c_int, bp, i32, vp, i32, vp, vp, u32, vp]
    lib.dpc_cluster.argtypes = [bp, i32, pp, vp, vp, vp, vp, u32, vp]
    lib.dpc_decision_graph.argtypes = [bp, vp, vp, i32, vp, vp, i32, i32, ctypes.c_double, vp, u32, vp]
    lib.dpc_priority_range.argtypes = [vp, ctypes.c_int, bp, vp, i32, vp, vp, vp, i32, vp, vp, u32, vp]
    lib.dpc_run.argtypes = [vp, ctypes.c_int, bp, pp, vp, vp, vp, vp, u32, vp]
    lib.dpc_run_host.argtypes = [vp, ctypes.c_int, bp, pp, vp, vp, vp, vp, u32, vp]
    lib.dpc_density_static.argtypes = [vp, ctypes.c_int, ctypes.c_int64, i32, ctypes.c_double, vp, u32, vp]
    lib.dpc_density_static.restype = ctypes.c_int
    lib.dpc_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.dpc_get_phase_times.argtypes = [vp, ctypes.POINTER(_PhaseTimes)]
    lib.dpc_get_phase_times.restype = ctypes.c_int
    lib.dpc_last_status.argtypes = [vp]
    lib.dpc_strerror.argtypes = [ctypes.c_int]
    lib.dpc_strerror.restype = ctypes.c_char_p
    lib.dpc_version.restype = ctypes.c_char_p
    lib.dpc_release.restype = None
    lib.dpc_cut_band.argtypes = [ctypes.c_double, i32, vp]
    lib.dpc_cut_band.restype = ctypes.c_int
    lib.dpc_probe_peak.argtypes = [ctypes.c_int, vp, vp]
    lib.dpc_probe_peak.restype = ctypes.c_int
    for f in ("dpc_density", "dpc_dependent", "dpc_cluster", "dpc_run", "dpc_run_host", "dpc_get_stats",
              "dpc_last_status"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().dpc_strerror(code).decode()
    except RuntimeError:
        return "status %d" % code


def version() -> str:
    return load().dpc_version().decode()


def cut_band(d_cut: float, dim: int):
    """(t_in, t_out, band_mul, band_add) of one cutoff: the float32
    certification band (dpc_cut_band; host arithmetic, no device)."""
    out = (ctypes.c_float * 4)()
    rc = load().dpc_cut_band(float(d_cut), int(dim), ctypes.cast(out, ctypes.c_void_p))
    if rc:
        raise DpcError(rc, "dpc_cut_band")
    return tuple(float(v) for v in out)


def probe_peak(kind: str = "fp32", stream=None) -> float:
    """Measured FMA throughput of this GPU in flop/s (dpc_probe_peak): "fp32"
    (FFMA) or "fp64" (DFMA)."""
    v = ctypes.c_double(0.0)
    _check(load().dpc_probe_peak({"fp32": 0, "fp64": 1}[kind], ctypes.cast(ctypes.pointer(v), ctypes.c_void_p),
                                 _stream(stream)), "dpc_probe_peak")
    return float(v.value)


def release() -> None:
    load().dpc_release()


# ---------------------------------------------------------------------------
# argument marshalling


class Batch:
    """Host-side batch descriptor (``dpc_batch``)."""

    def __init__(self, pt_offset: Sequence[int], dims: Sequence[int], d_cut, coord_offset=None):
        n_inst = len(dims)
        assert len(pt_offset) == n_inst + 1
        cuts = [[float(c) for c in (row if isinstance(row, (list, tuple)) else [row])] for row in d_cut]
        assert len(cuts) == n_inst and len({len(r) for r in cuts}) == 1
        self.n_inst = n_inst
        self.n_dcut = len(cuts[0])
        self.N = int(pt_offset[-1])
        self.dims = [int(d) for d in dims]
        self.pt_offset = [int(x) for x in pt_offset]
        self._po = (ctypes.c_int64 * (n_inst + 1))(*self.pt_offset)
        self._dim = (ctypes.c_int32 * n_inst)(*self.dims)
        self._dc = (ctypes.c_double * (n_inst * self.n_dcut))(*[c for r in cuts for c in r])
        self._co = (ctypes.c_int64 * n_inst)(*[int(x) for x in coord_offset]) if coord_offset is not None else None
        self.c = _Batch(n_inst, self._po, self._co, self._dim, self.n_dcut, self._dc)

    @classmethod
    def single(cls, n: int, d: int, d_cut) -> "Batch":
        cuts = list(d_cut) if isinstance(d_cut, (list, tuple)) else [d_cut]
        return cls([0, n], [d], [cuts])

    @classmethod
    def packed(cls, sizes: Sequence[int], dims: Sequence[int], d_cut) -> "Batch":
        po = [0]
        co = []
        c = 0
        for n, d in zip(sizes, dims):
            co.append(c)
            c += n * d
            po.append(po[-1] + n)
        return cls(po, dims, d_cut, coord_offset=co)

    @property
    def ptr(self):
        return ctypes.byref(self.c)


def make_params(batch: Batch, rho_noise, rho_min, delta_min):
    """``dpc_params`` array [n_inst * n_dcut]; scalars broadcast, lists per cutoff
    (length n_dcut) or per (instance, cutoff) (length n_inst * n_dcut)."""
    m = batch.n_inst * batch.n_dcut

    def expand(v):
        if isinstance(v, (list, tuple)):
            if len(v) == m:
                return list(v)
            if len(v) == batch.n_dcut:
                return list(v) * batch.n_inst
            raise ValueError("threshold list length %d" % len(v))
        return [v] * m
    rn, rm, dm = expand(rho_noise), expand(rho_min), expand(delta_min)
    arr = (_Params * m)(*[_Params(int(rn[i]), int(rm[i]), float(dm[i])) for i in range(m)])
    return arr


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return DPC_I32
    if t.dtype == torch.float32:
        return DPC_F32
    raise TypeError("points must be int32 or float32, got %s" % t.dtype)


def _dev(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _flags(precision: str, sync: bool, radius: int = 0, autotune: bool = False, layout: str = "auto") -> int:
    """Call flags: precision mode, synchronous status check, a fixed block
    radius (0 = default rule or autotuned choice), autotuning and a fixed
    kernel layout ("auto" = default rule or autotuned choice)."""
    return (PREC[precision] | (DPC_FLAG_SYNC_CHECK if sync else 0) | DPC_FLAG_RADIUS(radius)
            | (DPC_FLAG_AUTOTUNE if autotune else 0) | DPC_FLAG_LAYOUT(layout))


def _check(rc: int, what: str):
    if rc != DPC_OK:
        raise DpcError(rc, what)


def dpc_density(pts: torch.Tensor, batch: Batch, precision: str = "fp32", sync: bool = False,
                stream=None, out: torch.Tensor | None = None, autotune: bool = False,
                radius: int = 0, layout: str = "auto") -> torch.Tensor:
    lib = load()
    rho = out if out is not None else torch.empty((batch.n_dcut, batch.N), dtype=torch.int32, device=pts.device)
    _check(lib.dpc_density(_dev(pts, "pts"), _dtype_code(pts), batch.ptr, _dev(rho, "rho"),
                           _flags(precision, sync, radius, autotune, layout), _stream(stream)), "dpc_density")
    return rho


def dpc_dependent(pts: torch.Tensor, batch: Batch, dcut_index: int, rho: torch.Tensor, rho_skip: int = 0,
                  precision: str = "fp32", sync: bool = False, stream=None, radius: int = 0,
                  layout: str = "auto"):
    lib = load()
    if rho.dtype != torch.int32 or rho.numel() != batch.N:
        raise ValueError("rho must be int32 [N]")
    lam = torch.empty(batch.N, dtype=torch.int32, device=pts.device)
    delta = torch.empty(batch.N, dtype=torch.float64, device=pts.device)
    _check(lib.dpc_dependent(_dev(pts, "pts"), _dtype_code(pts), batch.ptr, int(dcut_index), _dev(rho, "rho"),
                             int(rho_skip), _dev(lam, "lambda"), _dev(delta, "delta"),
                             _flags(precision, sync, radius, False, layout), _stream(stream)), "dpc_dependent")
    return lam, delta


def dpc_cluster(batch: Batch, dcut_index: int, params, rho: torch.Tensor, lam: torch.Tensor, delta: torch.Tensor,
                sync: bool = False, stream=None) -> torch.Tensor:
    lib = load()
    label = torch.empty(batch.N, dtype=torch.int32, device=rho.device)
    _check(lib.dpc_cluster(batch.ptr, int(dcut_index), params, _dev(rho, "rho"), _dev(lam, "lambda"),
                           _dev(delta, "delta"), _dev(label, "label"), DPC_FLAG_SYNC_CHECK if sync else 0,
                           _stream(stream)), "dpc_cluster")
    return label


def dpc_decision_graph(batch: Batch, rho: torch.Tensor, delta: torch.Tensor, k: int = 16, rho_bins: int = 0,
                       delta_bins: int = 0, delta_lo: float = 1.0, sync: bool = False, stream=None) -> dict:
    """Decision-graph summaries of one cutoff: the top-k points by
    gamma = rho * delta per instance ("top" int32 [n_inst, k], "gamma" float64
    [n_inst, k]) and, with rho_bins/delta_bins > 0, the log2-binned (rho, delta)
    counts ("hist" int64 [n_inst, rho_bins, delta_bins])."""
    lib = load()
    if rho.dtype != torch.int32 or delta.dtype != torch.float64:
        raise ValueError("rho must be int32 and delta float64")
    dev = rho.device
    out = {}
    top = torch.empty((batch.n_inst, k), dtype=torch.int32, device=dev) if k > 0 else None
    gamma = torch.empty((batch.n_inst, k), dtype=torch.float64, device=dev) if k > 0 else None
    hist = (torch.empty((batch.n_inst, rho_bins, delta_bins), dtype=torch.int64, device=dev)
            if rho_bins > 0 and delta_bins > 0 else None)
    _check(lib.dpc_decision_graph(batch.ptr, _dev(rho, "rho"), _dev(delta, "delta"), int(k),
                                  _dev(top, "top") if top is not None else None,
                                  _dev(gamma, "gamma") if gamma is not None else None,
                                  int(rho_bins), int(delta_bins), float(delta_lo),
                                  _dev(hist, "hist") if hist is not None else None,
                                  DPC_FLAG_SYNC_CHECK if sync else 0, _stream(stream)), "dpc_decision_graph")
    if top is not None:
        out["top"], out["gamma"] = top, gamma
    if hist is not None:
        out["hist"] = hist
    return out


def range_boxes(lo, hi, device="cuda") -> torch.Tensor:
    """Query boxes [n, 2, 8] (float64) from lo, hi of shape [n, d] (d <= 8)."""
    lo = torch.as_tensor(lo, dtype=torch.float64)
    hi = torch.as_tensor(hi, dtype=torch.float64)
    if lo.dim() == 1:
        lo, hi = lo.reshape(-1, 1), hi.reshape(-1, 1)
    box = torch.zeros((lo.shape[0], 2, 8), dtype=torch.float64)
    box[:, 0, :lo.shape[1]] = lo
    box[:, 1, :hi.shape[1]] = hi
    return box.to(device)


def dpc_priority_range(pts: torch.Tensor, batch: Batch, rho: torch.Tensor, q_inst: torch.Tensor,
                       q_box: torch.Tensor, q_rho: torch.Tensor, max_out: int = 0, sync: bool = False,
                       stream=None) -> dict:
    """Priority range search: per query (instance q_inst, closed box q_box
    [n, 2, 8], threshold q_rho), "count" (int64 [n]) of the instance's points
    in the box with rho > q_rho and "ids" (int32 [n, max_out]): the smallest
    matching instance-local ids, ascending, padded with -1."""
    lib = load()
    if q_inst.dtype != torch.int32 or q_rho.dtype != torch.int32 or q_box.dtype != torch.float64:
        raise ValueError("q_inst and q_rho must be int32, q_box float64")
    nq = int(q_inst.numel())
    if tuple(q_box.shape) != (nq, 2, 8) or q_rho.numel() != nq:
        raise ValueError("q_box must be [n_query, 2, 8] and q_rho [n_query]")
    dev = rho.device
    count = torch.empty(nq, dtype=torch.int64, device=dev)
    ids = torch.empty((nq, max_out), dtype=torch.int32, device=dev) if max_out > 0 else None
    if nq:
        _check(lib.dpc_priority_range(_dev(pts, "pts"), _dtype_code(pts), batch.ptr, _dev(rho, "rho"), nq,
                                      _dev(q_inst, "q_inst"), _dev(q_box, "q_box"), _dev(q_rho, "q_rho"),
                                      int(max_out), _dev(count, "count"),
                                      _dev(ids, "ids") if ids is not None else None,
                                      DPC_FLAG_SYNC_CHECK if sync else 0, _stream(stream)), "dpc_priority_range")
    out = {"count": count}
    if ids is not None:
        out["ids"] = ids
    return out


def dpc_run(pts: torch.Tensor, batch: Batch, params, precision: str = "fp32", sync: bool = False, stream=None,
            out: dict | None = None, phase_times: bool = False, autotune: bool = False,
            radius: int = 0, graph: bool = False, layout: str = "auto", skip_noise: bool = False,
            near_shift: int = -1) -> dict:
    lib = load()
    shape = (batch.n_dcut, batch.N)
    if out is None:
        out = {"rho": torch.empty(shape, dtype=torch.int32, device=pts.device),
               "lam": torch.empty(shape, dtype=torch.int32, device=pts.device),
               "delta": torch.empty(shape, dtype=torch.float64, device=pts.device),
               "label": torch.empty(shape, dtype=torch.int32, device=pts.device)}
    _check(lib.dpc_run(_dev(pts, "pts"), _dtype_code(pts), batch.ptr, params, _dev(out["rho"], "rho"),
                       _dev(out["lam"], "lambda"), _dev(out["delta"], "delta"), _dev(out["label"], "label"),
                       _flags(precision, sync, radius, autotune, layout) | (DPC_FLAG_PHASE_TIMES if phase_times else 0)
                       | (DPC_FLAG_GRAPH if graph else 0) | (DPC_FLAG_SKIP_NOISE if skip_noise else 0)
                       | DPC_FLAG_NEAR_SHIFT(near_shift),
                       _stream(stream)),
           "dpc_run")
    return out


def dpc_run_host(pts: torch.Tensor, batch: Batch, params, precision: str = "fp32", stream=None,
                 out: dict | None = None, skip_noise: bool = False) -> dict:
    """Host-buffer form: `pts` and the results are CPU tensors (pin them for
    faster copies); the call returns after the results are on the host."""
    lib = load()
    if pts.is_cuda or not pts.is_contiguous():
        raise ValueError("pts must be a contiguous CPU tensor")
    shape = (batch.n_dcut, batch.N)
    if out is None:
        out = {"rho": torch.empty(shape, dtype=torch.int32), "lam": torch.empty(shape, dtype=torch.int32),
               "delta": torch.empty(shape, dtype=torch.float64), "label": torch.empty(shape, dtype=torch.int32)}

    def hp(t):
        return ctypes.c_void_p(t.data_ptr())
    _check(lib.dpc_run_host(hp(pts), _dtype_code(pts), batch.ptr, params, hp(out["rho"]), hp(out["lam"]),
                            hp(out["delta"]), hp(out["label"]),
                            _flags(precision, True) | (DPC_FLAG_SKIP_NOISE if skip_noise else 0), _stream(stream)),
           "dpc_run_host")
    return out


def dpc_get_stats(stream=None) -> dict:
    lib = load()
    s = _Stats()
    _check(lib.dpc_get_stats(_stream(stream), ctypes.byref(s)), "dpc_get_stats")
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def dpc_density_static(pts: torch.Tensor, d_cut: float, precision: str = "fp32", sync: bool = False,
                       stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Densities of one point set ``pts`` [n, d] with the library's fixed
    scratch area (no device allocation inside the call; see dpc.h)."""
    lib = load()
    if pts.dim() == 1:
        pts = pts.reshape(-1, 1)
    n, d = pts.shape
    rho = out if out is not None else torch.empty(n, dtype=torch.int32, device=pts.device)
    _check(lib.dpc_density_static(_dev(pts, "pts"), _dtype_code(pts), n, d, float(d_cut), _dev(rho, "rho"),
                                  _flags(precision, sync), _stream(stream)), "dpc_density_static")
    return rho


def dpc_get_phase_times(stream=None) -> dict:
    """{phase: (milliseconds, launches)} of the last call made with phase times."""
    lib = load()
    t = _PhaseTimes()
    _check(lib.dpc_get_phase_times(_stream(stream), ctypes.byref(t)), "dpc_get_phase_times")
    return {p: (t.ms[i], t.launches[i]) for i, p in enumerate(PHASES)}


def dpc_last_status(stream=None) -> int:
    return load().dpc_last_status(_stream(stream))


# ---------------------------------------------------------------------------
# convenience


def run(pts: torch.Tensor, d_cut, rho_noise, rho_min, delta_min, precision: str = "fp32", sync: bool = True,
        stream=None, autotune: bool = False, radius: int = 0, layout: str = "auto",
        skip_noise: bool = False, near_shift: int = -1) -> dict:
    """DPC of one point set ``pts`` [n, d] (CUDA, int32/float32) for one or more cutoffs."""
    if pts.dim() == 1:
        pts = pts.reshape(-1, 1)
    n, d = pts.shape
    cuts = list(d_cut) if isinstance(d_cut, (list, tuple)) else [d_cut]
    batch = Batch.single(n, d, cuts)
    params = make_params(batch, rho_noise, rho_min, delta_min)
    return dpc_run(pts.contiguous(), batch, params, precision=precision, sync=sync, stream=stream,
                   autotune=autotune, radius=radius, layout=layout, skip_noise=skip_noise,
                   near_shift=near_shift)

