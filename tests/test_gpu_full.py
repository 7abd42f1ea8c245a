"""GPU parity at the full workload sizes (1e6 to 1e7 points).

The oracle cannot evaluate every point of these sets (O(n^2)), so each test
  * compares seeded sample points one by one with the oracle's per-point
    forms (density from the definition; dependent point by walking candidates
    in distance order with densities computed from scratch), bit for bit;
  * checks properties that hold at any size on every point: delta is the
    canonical binary64 distance to lambda, lambda is higher in the order, one
    top point per cutoff, labels form the forest the definitions describe;
  * checks that the float32-certified and the plain binary64 paths agree
    byte for byte.
The launch configuration is the one bench.py times (dpc_run, all cutoffs).
"""
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


def run(w, precision):
    t = torch.from_numpy(w.pts).cuda()
    batch = dpc.Batch.single(w.n, w.d, w.d_cut)
    params = dpc.make_params(batch, w.rho_noise, w.rho_min, w.delta_min)
    out = dpc.dpc_run(t, batch, params, precision=precision, sync=True)
    return {k: v.cpu().numpy() for k, v in out.items()}


def canonical_s64(pts, i, j):
    """The binary64 squared distance, coordinates in increasing order, numpy
    elementwise (round to nearest, no contraction)."""
    x = pts.astype(np.float64)
    s = np.zeros(len(i), np.float64)
    for k in range(pts.shape[1]):
        t = x[i, k] - x[j, k]
        s = s + t * t
    return s


def check_properties(w, out, c):
    rho, lam, delta, lab = out["rho"][c], out["lam"][c], out["delta"][c], out["label"][c]
    n = w.n
    ids = np.arange(n)
    assert rho.min() >= 1
    assert (int(rho.sum()) - n) % 2 == 0
    root = np.flatnonzero(lam < 0)
    assert len(root) == 1, "exactly one point without a dependent point"
    r = root[0]
    assert np.isinf(delta[r]) and rho[r] == rho.max() and r == np.flatnonzero(rho == rho.max()).min()
    nr = lam >= 0
    hi = (rho[lam[nr]] > rho[nr]) | ((rho[lam[nr]] == rho[nr]) & (lam[nr] < ids[nr]))
    assert hi.all(), "dependent points are higher in the order"
    s = canonical_s64(w.pts, ids[nr], lam[nr])
    assert np.array_equal(np.sqrt(s).view(np.int64), delta[nr].view(np.int64)), "delta = D(x, lambda)"
    noise = rho < w.rho_noise[c]
    center = ~noise & ((lam < 0) | ((rho >= w.rho_min[c]) & (delta >= w.delta_min[c])))
    assert np.array_equal(lab == -1, noise)
    assert np.array_equal(lab[center], ids[center])
    rest = ~noise & ~center
    assert np.array_equal(lab[rest], lab[lam[rest]])


def check_samples(w, out, c, m, extra_ids, seed, min_resolved=0.8, max_checks=48):
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([rng.choice(w.n, m, replace=False), extra_ids])).astype(np.int64)
    rho_o = oracle.density(w.pts, w.d_cut[c], idx=idx)
    assert np.array_equal(out["rho"][c][idx], rho_o), "sampled densities"
    lam_o, delta_o, rho2, ok = oracle.dependent_at(w.pts, w.d_cut[c], idx, max_checks=max_checks)
    assert np.array_equal(rho2, rho_o)
    assert ok.mean() >= min_resolved, ok.mean()
    assert np.array_equal(out["lam"][c][idx[ok]], lam_o[ok]), "sampled dependent points"
    assert np.array_equal(out["delta"][c][idx[ok]].view(np.int64), delta_o[ok].view(np.int64))
    return int(ok.sum())


def test_c2_full():
    w = W.c2()
    f32 = run(w, "fp32")
    check_properties(w, f32, 0)
    check_samples(w, f32, 0, 256, w.noise_ids[:32], 21)
    f64 = run(w, "fp64")
    for k in f32:
        assert np.array_equal(f32[k].view(np.uint8), f64[k].view(np.uint8)), k


def test_c3_full():
    w = W.c3()
    out = run(w, "fp32")
    check_properties(w, out, 0)
    check_samples(w, out, 0, 96, w.noise_ids[:16], 31, max_checks=24)


def test_c5_full_sweep():
    w = W.c5()
    out = run(w, "fp32")
    for c in range(len(w.d_cut)):
        check_properties(w, out, c)
        assert np.all(out["rho"][c] >= out["rho"][c - 1]) if c else True  # rho grows with d_cut
    check_samples(w, out, 0, 96, w.noise_ids[:16], 51, max_checks=24)
    check_samples(w, out, 3, 48, w.noise_ids[16:24], 52, max_checks=24)


def test_c4_full_batch():
    """The 4096-instance batch with 8 cutoffs each, in one dpc_run (the call
    bench.py times).  The 8 smallest instances are compared with the oracle in
    full for every cutoff; 40 random instances get the whole-instance
    properties and sampled oracle checks at the first and last cutoff."""
    from types import SimpleNamespace
    from _gpu_util import assert_same

    w = W.c4()
    batch = dpc.Batch([0] + list(np.cumsum(w.sizes)), w.dims, w.d_cut, coord_offset=w.coord_offset)
    params = dpc.make_params(batch, w.rho_noise, w.rho_min, w.delta_min)
    out = dpc.dpc_run(torch.from_numpy(w.flat).cuda(), batch, params, sync=True)
    po = batch.pt_offset
    ncut = batch.n_dcut

    def inst_out(i):
        return {k: v[:, po[i]:po[i + 1]].cpu().numpy() for k, v in out.items()}

    order = np.argsort(w.sizes, kind="stable")
    for i in order[:8]:
        got = inst_out(i)
        pts = w.instance(i)
        for c in range(ncut):
            j = i * ncut + c
            ref = oracle.run(pts, w.d_cut[i][c], w.rho_noise[j], w.rho_min[j], w.delta_min[j])
            assert_same({k: v[c] for k, v in got.items()}, ref, "instance %d cut %d" % (i, c))
    rng = np.random.default_rng(41)
    for i in rng.choice(len(w.sizes), 40, replace=False):
        got = inst_out(i)
        view = SimpleNamespace(pts=w.instance(i), n=w.sizes[i], d_cut=w.d_cut[i],
                               rho_noise=w.rho_noise[i * ncut:(i + 1) * ncut],
                               rho_min=w.rho_min[i * ncut:(i + 1) * ncut],
                               delta_min=w.delta_min[i * ncut:(i + 1) * ncut])
        for c in (0, ncut - 1):
            check_properties(view, got, c)
            check_samples(view, got, c, 12, np.zeros(0, np.int64), 4100 + int(i), min_resolved=0.5,
                          max_checks=32)
