"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle,
element by element, on seeded inputs that span many grid cells and tiles,
plus the edge cases the method has.  Both precision modes must give the
oracle's exact output (see _gpu_util for the tolerance: none)."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2305_11335_gb300 as dpc
import workloads as W
from _gpu_util import assert_same, bits, gpu_run, parity

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("name", ["hand_example_1d.json", "hand_example_2d.json"])
@pytest.mark.parametrize("dtype,scale", [(np.int32, 1.0), (np.float32, 0.25)])
def test_hand_examples(name, dtype, scale):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    pts = np.ascontiguousarray((np.array(g["points"], np.float64) * scale).astype(dtype))
    got = gpu_run(pts, [g["d_cut"] * scale], g["rho_noise"], g["rho_min"], g["delta_min"] * scale)
    assert got["rho"][0].tolist() == g["rho"]
    assert got["lam"][0].tolist() == g["lambda"]
    want = [math.inf if v == "inf" else v * scale for v in g["delta"]]
    assert got["delta"][0].tolist() == want
    assert got["label"][0].tolist() == g["label"]


@pytest.mark.parametrize("dim,k", [(1, 40), (2, 23), (3, 9)])
def test_lattices(dim, k):
    pts = W.lattice(k, dim, 1)
    parity(pts, [1.0, math.sqrt(2.0), np.nextafter(1.0, 0.0), 2.0], rho_noise=1, rho_min=2, delta_min=1.5)


def test_line_deep_chain():
    pts = W.line(5000, np.int32)
    parity(pts, [1.0, 3.0], rho_noise=1, rho_min=1, delta_min=10.0)


@pytest.mark.parametrize("n,d", [(17, 3), (300, 8), (1, 2), (2, 5)])
def test_all_equal_and_tiny(n, d):
    pts = W.all_equal(n, d)
    parity(pts, [0.0, 1.0], rho_noise=1, rho_min=1, delta_min=0.5)


def test_zero_and_huge_cutoff():
    pts = W.random_blobs(2000, 2, 31, dtype=np.float32, dup_frac=0.05)
    parity(pts, [0.0, 1e-6, 50.0], rho_noise=1, rho_min=2, delta_min=0.05)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 8])
@pytest.mark.parametrize("dtype", [np.float32, np.int32])
def test_random_blobs(d, dtype):
    n = 6000 if d <= 3 else 3000
    scale = 2000.0 if dtype == np.int32 else 1.0
    pts = W.random_blobs(n, d, 100 + d, dtype=dtype, scale=scale, dup_frac=0.02)
    dc = 0.03 * scale * (1.0 + 0.6 * (d - 1))
    parity(pts, [dc, 1.5 * dc], rho_noise=3, rho_min=8, delta_min=4 * dc)


def test_c1_full():
    w = W.c1()
    parity(w.pts, w.d_cut, w.rho_noise[0], w.rho_min[0], w.delta_min[0])


def test_boundary_band():
    """Pairs at exactly d_cut and one float step either side: the float32
    filter cannot decide them, the binary64 recheck must."""
    rng = np.random.default_rng(5)
    base = rng.random((400, 3)) * 10.0
    dc = 0.37
    u = rng.standard_normal((400, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    partner = base + dc * u
    pts = np.concatenate([base, partner]).astype(np.float32)
    # nudge partners by single float steps in random directions
    k = rng.integers(-2, 3, (400, 3))
    for s in range(3):
        pts[400:, s] = np.array([np.nextafter(np.float32(v), np.float32(np.sign(t) * np.inf)) if t else v
                                 for v, t in zip(pts[400:, s], k[:, s])], np.float32)
    parity(pts, [dc], rho_noise=1, rho_min=2, delta_min=1.0)


def test_large_offset_cancellation():
    """Coordinates near 1e5 with tiny spreads: float32 differences cancel."""
    rng = np.random.default_rng(9)
    pts = (1e5 + rng.random((3000, 2)) * 0.5).astype(np.float32)
    parity(pts, [0.01, 0.003], rho_noise=1, rho_min=2, delta_min=0.05)


def test_equidistant_ties_int():
    """Integer points on a coarse lattice with random duplicates: many exact
    distance ties, decided by the smaller id."""
    rng = np.random.default_rng(3)
    pts = rng.integers(0, 40, (5000, 2)).astype(np.int32)
    parity(pts, [1.0, 2.0, 2.5], rho_noise=2, rho_min=4, delta_min=3.0)


def test_batched_equals_single():
    sizes = [500, 1, 0, 2500, 1200]
    dims = [2, 3, 2, 5, 1]
    insts = [W.random_blobs(n, d, 200 + i) if n else np.zeros((0, d), np.float32)
             for i, (n, d) in enumerate(zip(sizes, dims))]
    cuts = [[0.02 * (1 + 0.5 * (d - 1)), 0.04 * (1 + 0.5 * (d - 1))] for d in dims]
    batch = dpc.Batch.packed(sizes, dims, cuts)
    flat = torch.from_numpy(np.concatenate([p.reshape(-1) for p in insts]).astype(np.float32)).cuda()
    params = dpc.make_params(batch, 2, 3, [0.1] * (len(sizes) * 2))
    out = dpc.dpc_run(flat, batch, params, sync=True)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    for i, p in enumerate(insts):
        lo, hi = batch.pt_offset[i], batch.pt_offset[i + 1]
        for c in range(2):
            ref = oracle.run(p, cuts[i][c], 2, 3, 0.1)
            assert_same({k: v[c, lo:hi] for k, v in out.items()}, ref, "inst %d cut %d" % (i, c))


def test_split_entry_points_match_run():
    pts = W.random_blobs(4000, 3, 77)
    dc = 0.05
    t = torch.from_numpy(pts).cuda()
    batch = dpc.Batch.single(4000, 3, [dc])
    params = dpc.make_params(batch, 3, 6, 0.2)
    rho = dpc.dpc_density(t, batch, sync=True)
    lam, delta = dpc.dpc_dependent(t, batch, 0, rho[0].contiguous(), sync=True)
    label = dpc.dpc_cluster(batch, 0, params, rho[0].contiguous(), lam, delta, sync=True)
    ref = oracle.run(pts, dc, 3, 6, 0.2)
    assert_same({"rho": rho[0].cpu().numpy(), "lam": lam.cpu().numpy(), "delta": delta.cpu().numpy(),
                 "label": label.cpu().numpy()}, ref)


def test_dependent_accepts_any_rho():
    """dpc_dependent is a function of (points, rho): feed it densities that
    are not those of any cutoff (seeded random), with a noise skip."""
    pts = W.random_blobs(3000, 2, 55)
    rng = np.random.default_rng(1)
    rho = rng.integers(1, 12, 3000).astype(np.int32)
    t = torch.from_numpy(pts).cuda()
    batch = dpc.Batch.single(3000, 2, [0.02])
    for prec in ("fp32", "fp64"):
        lam, delta = dpc.dpc_dependent(t, batch, 0, torch.from_numpy(rho).cuda(), rho_skip=3, precision=prec,
                                       sync=True)
        rl, rd = oracle.dependent(pts, rho, rho_skip=3)
        assert np.array_equal(lam.cpu().numpy(), rl)
        assert np.array_equal(bits(delta.cpu().numpy()), bits(rd))


def test_cluster_on_generated_forest():
    """dpc_cluster on a seeded random forest (lambda pointing to higher ids
    in a random order) with thresholds that create noise and centers."""
    rng = np.random.default_rng(8)
    n = 20000
    order = rng.permutation(n)           # order[0] is the highest point
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    rho = (n - rank).astype(np.int32) // 50 + 1
    lam = np.full(n, -1, np.int32)
    for r in range(1, n):
        lam[order[r]] = order[rng.integers(max(0, r - 40), r)]
    delta = rng.random(n) * 10.0
    delta[order[0]] = np.inf
    ref = oracle.cluster(rho, lam, delta, 20, 60, 8.5)
    batch = dpc.Batch.single(n, 2, [1.0])
    params = dpc.make_params(batch, 20, 60, 8.5)
    got = dpc.dpc_cluster(batch, 0, params, torch.from_numpy(rho).cuda(), torch.from_numpy(lam).cuda(),
                          torch.from_numpy(delta).cuda(), sync=True)
    assert np.array_equal(got.cpu().numpy(), ref)


def test_cluster_reports_cycles():
    """Dependent pointers that do not form a forest (a three-cycle, with a long
    chain leading into it) are reported as DPC_ERR_DATA, and a forest
    afterwards is labelled exactly."""
    n = 5000
    rho = np.full(n, 10, np.int32)
    lam = (np.arange(n) - 1).astype(np.int32)   # i depends on i - 1
    lam[0] = -1
    delta = np.full(n, 1.0)
    delta[0] = np.inf
    batch = dpc.Batch.single(n, 2, [1.0])
    params = dpc.make_params(batch, 1, 5, 5.0)
    ref = oracle.cluster(rho, lam, delta, 1, 5, 5.0)
    cyc = lam.copy()
    cyc[10], cyc[11], cyc[12] = 12, 10, 11      # 10 -> 12 -> 11 -> 10; 13.. lead into it
    with pytest.raises(dpc.DpcError) as e:
        dpc.dpc_cluster(batch, 0, params, torch.from_numpy(rho).cuda(), torch.from_numpy(cyc).cuda(),
                        torch.from_numpy(delta).cuda(), sync=True)
    assert e.value.code == dpc.DPC_ERR_DATA
    got = dpc.dpc_cluster(batch, 0, params, torch.from_numpy(rho).cuda(), torch.from_numpy(lam).cuda(),
                          torch.from_numpy(delta).cuda(), sync=True)
    assert np.array_equal(got.cpu().numpy(), ref)
    assert np.all(ref == 0)


def test_bad_coordinates_reported():
    pts = W.random_blobs(100, 2, 4)
    pts[17, 1] = np.nan
    with pytest.raises(dpc.DpcError) as e:
        gpu_run(pts, [0.1], 1, 1, 1.0)
    assert e.value.code == dpc.DPC_ERR_DATA
    ip = W.random_blobs(100, 2, 4, dtype=np.int32, scale=100.0)
    ip[3, 0] = (1 << 24) + 1
    with pytest.raises(dpc.DpcError) as e:
        gpu_run(ip, [5.0], 1, 1, 1.0)
    assert e.value.code == dpc.DPC_ERR_DATA
    # the library recovers: a valid call afterwards succeeds
    parity(W.random_blobs(300, 2, 4), [0.05], precisions=("fp32",))


def test_repeat_runs_identical():
    pts = W.random_blobs(20000, 3, 66)
    outs = [gpu_run(pts, [0.04], 3, 6, 0.2) for _ in range(3)]
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k].view(np.uint8), outs[0][k].view(np.uint8))


def test_run_host_matches_device():
    pts = W.random_blobs(5000, 2, 12)
    batch = dpc.Batch.single(5000, 2, [0.02, 0.03])
    params = dpc.make_params(batch, 2, 4, 0.1)
    host = dpc.dpc_run_host(torch.from_numpy(pts).pin_memory(), batch, params)
    dev = dpc.dpc_run(torch.from_numpy(pts).cuda(), batch, params, sync=True)
    for k in host:
        assert np.array_equal(host[k].numpy().view(np.uint8), dev[k].cpu().numpy().view(np.uint8))


def test_run_host_batch_matches_oracle():
    """The host-buffer entry point copies each output back as soon as its
    phase has finished for the last dimension class; a batch of several
    classes and two cutoffs checks that every per-cutoff copy holds the
    finished values (against the oracle), twice in a row."""
    sizes = [700, 0, 2100, 900, 1300]
    dims = [2, 3, 3, 5, 1]
    insts = [W.random_blobs(n, d, 300 + i) if n else np.zeros((0, d), np.float32)
             for i, (n, d) in enumerate(zip(sizes, dims))]
    cuts = [[0.02 * (1 + 0.5 * (d - 1)), 0.04 * (1 + 0.5 * (d - 1))] for d in dims]
    batch = dpc.Batch.packed(sizes, dims, cuts)
    flat = torch.from_numpy(np.concatenate([q.reshape(-1) for q in insts]).astype(np.float32))
    params = dpc.make_params(batch, 2, 3, [0.1] * (len(sizes) * 2))
    for _ in range(2):
        out = dpc.dpc_run_host(flat.pin_memory(), batch, params)
        out = {k: v.numpy() for k, v in out.items()}
        for i, q in enumerate(insts):
            lo, hi = batch.pt_offset[i], batch.pt_offset[i + 1]
            for c in range(2):
                ref = oracle.run(q, cuts[i][c], 2, 3, 0.1)
                assert_same({k: v[c, lo:hi] for k, v in out.items()}, ref, "inst %d cut %d" % (i, c))


def test_stats():
    pts = W.random_blobs(20000, 2, 67)
    gpu_run(pts, [0.01], 2, 4, 0.1)
    s = dpc.dpc_get_stats()
    assert s["occupied_cells"] > 0 and s["bits_per_axis"] >= 1
    assert 0 < s["far_queries"] < 20000


@pytest.mark.parametrize("layout", ["union", "segment", "tree", "tensor", "pairs", "cell"])
@pytest.mark.parametrize("radius", [1, 2, 3, 5])
def test_block_radius_does_not_change_results(radius, layout):
    """Every block radius (grid level) and both kernel layouts give the
    oracle's result, in 1, 2, 3 and 5 dimensions (radii above a dimension's
    maximum are clamped)."""
    for d, n, dc in ((1, 3000, 0.004), (2, 4000, 0.03), (3, 4000, 0.06), (5, 2500, 0.12)):
        pts = W.random_blobs(n, d, 900 + d)
        refs = [oracle.run(pts, c, 2, 3, 0.1) for c in (dc, dc * 1.3)]
        t = torch.from_numpy(pts).cuda()
        out = dpc.run(t, [dc, dc * 1.3], 2, 3, 0.1, radius=radius, layout=layout)
        for c, ref in enumerate(refs):
            assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref, "d=%d r=%d cut %d" % (d, radius, c))
        st = dpc.dpc_get_stats()
        assert 1 <= st["block_radius"] <= (5 if d <= 2 else (2 if d == 3 else 1))


@pytest.mark.parametrize("layout", ["union", "segment", "cell"])
@pytest.mark.parametrize("shift", [0, 1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_near_shift_does_not_change_results(shift, layout, precision):
    """The near phase on cells one or two levels finer than the density's
    (more queries left to the tree search) gives the oracle's result."""
    rng = np.random.default_rng(77)
    cases = [(W.random_blobs(4000, 2, 950), 0.03), (W.random_blobs(4000, 3, 951), 0.06),
             (W.random_blobs(2500, 5, 952), 0.12), (rng.integers(0, 40, (3000, 2)).astype(np.int32), 2.0)]
    for pts, dc in cases:
        refs = [oracle.run(pts, c, 2, 3, 0.1) for c in (dc, dc * 1.3)]
        t = torch.from_numpy(pts).cuda()
        out = dpc.run(t, [dc, dc * 1.3], 2, 3, 0.1, layout=layout, near_shift=shift, precision=precision)
        for c, ref in enumerate(refs):
            assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref,
                        "d=%d shift=%d cut %d" % (pts.shape[1], shift, c))
        assert dpc.dpc_get_stats()["near_shift"] == shift


def test_autotune_keeps_results_and_caches():
    pts = W.random_blobs(20000, 2, 4242)
    dc = 0.01
    ref = oracle.run(pts, dc, 2, 3, 0.1)
    t = torch.from_numpy(pts).cuda()
    first = dpc.run(t, [dc], 2, 3, 0.1, autotune=True)
    r1 = dpc.dpc_get_stats()["block_radius"]
    again = dpc.run(t, [dc], 2, 3, 0.1)
    r2 = dpc.dpc_get_stats()["block_radius"]
    assert r1 == r2 and 1 <= r1 <= 3
    for out in (first, again):
        assert_same({k: v[0].cpu().numpy() for k, v in out.items()}, ref)


def test_graph_mode_replays_and_recaptures():
    """DPC_FLAG_GRAPH: capture on the first call, replay on identical calls
    (new coordinates in the same buffer are picked up), capture again when
    the batch changes; every result equals the oracle's."""
    s = torch.cuda.Stream()
    n, d = 6000, 2
    sets = [W.random_blobs(n, d, 7100 + i) for i in range(3)]
    t = torch.from_numpy(sets[0]).cuda()
    torch.cuda.synchronize()
    for cuts in ([0.02, 0.03], [0.025]):
        batch = dpc.Batch.single(n, d, cuts)
        params = dpc.make_params(batch, 2, 3, 0.1)
        out = {"rho": torch.empty((len(cuts), n), dtype=torch.int32, device="cuda"),
               "lam": torch.empty((len(cuts), n), dtype=torch.int32, device="cuda"),
               "delta": torch.empty((len(cuts), n), dtype=torch.float64, device="cuda"),
               "label": torch.empty((len(cuts), n), dtype=torch.int32, device="cuda")}
        for rep, pts in enumerate(sets):
            with torch.cuda.stream(s):
                t.copy_(torch.from_numpy(pts))
                dpc.dpc_run(t, batch, params, stream=s, out=out, graph=True, sync=True)
            for c, dc in enumerate(cuts):
                ref = oracle.run(pts, dc, 2, 3, 0.1)
                assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref,
                            "cuts %r rep %d cut %d" % (cuts, rep, c))
    assert dpc.dpc_get_stats(s)["kernel_launches"] > 10


def test_graph_mode_batch():
    """A multi-class batch in graph mode: the instance tables are copied before
    every replay."""
    s = torch.cuda.Stream()
    sizes, dims = [300, 0, 1, 900, 45, 2000, 64], [2, 3, 3, 5, 2, 3, 7]
    insts = [W.random_blobs(nn, dd, 7300 + i) if nn else np.zeros((0, dd), np.float32)
             for i, (nn, dd) in enumerate(zip(sizes, dims))]
    cuts = [[0.05 * (1 + 0.3 * (dd - 1))] for dd in dims]
    batch = dpc.Batch.packed(sizes, dims, cuts)
    params = dpc.make_params(batch, 2, 3, 0.1)
    t = torch.from_numpy(np.concatenate([p.reshape(-1) for p in insts]).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    for rep in range(3):
        with torch.cuda.stream(s):
            out = dpc.dpc_run(t, batch, params, stream=s, graph=True, sync=True)
        out = {k: v.cpu().numpy() for k, v in out.items()}
        for i, p in enumerate(insts):
            lo, hi = batch.pt_offset[i], batch.pt_offset[i + 1]
            ref = oracle.run(p, cuts[i][0], 2, 3, 0.1)
            assert_same({k: v[0, lo:hi] for k, v in out.items()}, ref, "rep %d inst %d" % (rep, i))


@pytest.mark.parametrize("d,dtype", [(5, np.float32), (6, np.float32), (8, np.float32), (5, np.int32)])
def test_tensor_density_dense_blocks(d, dtype):
    """The tensor-core density in 5-8 dimensions on dense blocks (many 256-
    candidate tiles per segment, 128-point items over several cells) and, for
    integer coordinates, many pairs exactly at the cutoff (the error band and
    its binary64 recount decide them)."""
    rng = np.random.default_rng(300 + d)
    if dtype == np.int32:
        pts = rng.integers(0, 12, (12000, d)).astype(np.int32)
        cuts = [3.0, 4.0]
    else:
        pts = W.random_blobs(12000, d, 310 + d, n_blobs=3)
        cuts = [0.15, 0.25]
    t = torch.from_numpy(pts).cuda()
    for c in cuts:
        ref = oracle.density(pts, c)
        for prec in ("fp32", "fp64"):
            got = dpc.dpc_density(t, dpc.Batch.single(len(pts), d, [c]), precision=prec, sync=True,
                                  layout="tensor")
            assert np.array_equal(got[0].cpu().numpy(), ref), (d, c, prec)
            # the tensor cores ran the float32 call; binary64 falls back to segments
            assert dpc.dpc_get_stats()["density_layout"] == (4 if prec == "fp32" else 2), prec


@pytest.mark.parametrize("d,dtype", [(5, np.float32), (7, np.float32), (8, np.float32), (5, np.int32),
                                     (6, np.int32)])
def test_tensor_near_phase(d, dtype):
    """The tensor-core near phase (and density) in 5-8 dimensions: dense blocks
    of many 256-candidate tiles, and for integer coordinates many exactly equal
    distances (candidates no bound separates go to the far phase, which ranks
    them in binary64); every output against the oracle, and the near phase
    checked to have run on the tensor cores."""
    rng = np.random.default_rng(500 + d)
    if dtype == np.int32:
        pts = rng.integers(0, 9, (8000, d)).astype(np.int32)
        cuts = [2.0, 3.0]
    else:
        pts = W.random_blobs(10000, d, 510 + d, n_blobs=3, dup_frac=0.01)
        cuts = [0.12, 0.2]
    refs = [oracle.run(pts, c, 2, 3, 0.1) for c in cuts]
    t = torch.from_numpy(pts).cuda()
    out = dpc.run(t, cuts, 2, 3, 0.1, layout="tensor")
    st = dpc.dpc_get_stats()
    assert st["near_layout"] == 4 and st["density_layout"] == 4
    for c, ref in enumerate(refs):
        assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref, "d=%d cut %d" % (d, c))


@pytest.mark.parametrize("d,dtype", [(1, np.int32), (2, np.float32), (2, np.int32), (3, np.float32),
                                     (3, np.int32), (4, np.float32), (6, np.float32)])
def test_cell_layout_large_cells(d, dtype):
    """The cell layout where cells hold more queries than a warp has lanes
    (several queries per lane, several passes) and blocks hold more candidates
    than one shared-memory window (several windows), with exact integer ties
    at the cutoff, in both precision modes."""
    rng = np.random.default_rng(400 + d)
    if dtype == np.int32:
        side = {1: 4000, 2: 60, 3: 16}.get(d, 8)
        pts = rng.integers(0, side, (20000, d)).astype(np.int32)
        cuts = [2.0, 3.0] if d > 1 else [5.0, 40.0]
    else:
        pts = W.random_blobs(20000, d, 410 + d, n_blobs=2, dup_frac=0.01)
        cuts = [0.05 * d ** 0.5, 0.1 * d ** 0.5]
    refs = [oracle.run(pts, c, 2, 3, 0.1) for c in cuts]
    t = torch.from_numpy(pts).cuda()
    for prec in ("fp32", "fp64"):
        out = dpc.run(t, cuts, 2, 3, 0.1, layout="cell", precision=prec)
        st = dpc.dpc_get_stats()
        assert st["density_layout"] == 6 and st["near_layout"] == 6
        for c, ref in enumerate(refs):
            assert_same({k: v[c].cpu().numpy() for k, v in out.items()}, ref, "%s d=%d cut %d" % (prec, d, c))
