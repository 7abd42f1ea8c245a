"""Pins for the CPU oracle: facts fixed by the paper's definitions and by
mathematics, each checked against something other than the oracle itself.

Every pin takes the oracle ``variant`` so that ``test_oracle.py`` can show each
planted mistake (a deviation from Definitions 1-5 or from a fixed reading) is
caught by at least one pin.  A pin returns None when it holds and raises
AssertionError otherwise.
"""
import json
import math
import os

import numpy as np

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _as_dtype(pts, dtype):
    return np.ascontiguousarray(np.asarray(pts).astype(dtype))


def _golden_delta(vals):
    return np.array([math.inf if v == "inf" else float(v) for v in vals], dtype=np.float64)


# --- worked examples ---------------------------------------------------------


def pin_hand_examples(variant=0):
    """The hand-worked examples in tests/golden (Definitions 1-5)."""
    for name in ("hand_example_1d.json", "hand_example_2d.json"):
        with open(os.path.join(GOLDEN, name)) as f:
            g = json.load(f)
        base = np.array(g["points"], dtype=np.int64)
        # the same example in float32, scaled by 1/4 (exact in binary32 and binary64)
        for dtype, scale in ((np.int32, 1.0), (np.float32, 0.25)):
            pts = _as_dtype(base * scale, dtype)
            dc = g["d_cut"] * scale
            rho = oracle.density(pts, dc, variant=variant)
            assert np.array_equal(rho, g["rho"]), (name, dtype, rho)
            lam, delta = oracle.dependent(pts, rho, variant=variant)
            assert np.array_equal(lam, g["lambda"]), (name, dtype, lam)
            assert np.array_equal(delta, _golden_delta(g["delta"]) * scale), (name, dtype, delta)
            lab = oracle.cluster(rho, lam, delta, g["rho_noise"], g["rho_min"], g["delta_min"] * scale,
                                 variant=variant)
            assert np.array_equal(lab, g["label"]), (name, dtype, lab)


# --- closed forms for rho ----------------------------------------------------


def pin_lattice_2d(variant=0):
    """k x k unit lattice.  d_cut = 1: interior 5, edge 4, corner 3.
    d_cut = sqrt(2): interior 9, edge 6, corner 4.  d_cut just below 1: 1."""
    k = 7
    for dtype, spacing in ((np.int32, 1), (np.float32, 0.25)):
        pts = _as_dtype(W.lattice(k, 2, 1).astype(np.float64) * spacing, dtype)
        ij = W.lattice(k, 2, 1)
        border = (ij == 0) | (ij == k - 1)
        nb = border.sum(axis=1)  # 0 interior, 1 edge, 2 corner
        rho = oracle.density(pts, 1.0 * spacing, variant=variant)
        assert np.array_equal(rho, np.choose(nb, [5, 4, 3])), (dtype, rho)
        rho = oracle.density(pts, math.sqrt(2.0) * spacing, variant=variant)
        assert np.array_equal(rho, np.choose(nb, [9, 6, 4])), (dtype, rho)
        rho = oracle.density(pts, np.nextafter(1.0, 0.0) * spacing, variant=variant)
        assert np.all(rho == 1), (dtype, rho)


def pin_lattice_3d(variant=0):
    """k^3 unit lattice, d_cut = 1: 1 + number of axis neighbours, i.e.
    7 interior, 6 face, 5 edge, 4 corner."""
    k = 5
    ij = W.lattice(k, 3, 1)
    border = ((ij == 0) | (ij == k - 1)).sum(axis=1)
    for dtype in (np.int32, np.float32):
        pts = _as_dtype(ij, dtype)
        rho = oracle.density(pts, 1.0, variant=variant)
        assert np.array_equal(rho, 7 - border), rho


def pin_all_equal(variant=0):
    """n identical points: rho = n; the lowest id is the highest point; every
    other point depends on id 0 at distance 0."""
    for n, d in ((17, 3), (5, 1), (9, 8)):
        pts = W.all_equal(n, d)
        rho = oracle.density(pts, 0.0, variant=variant)
        assert np.all(rho == n), rho
        lam, delta = oracle.dependent(pts, rho, variant=variant)
        assert lam[0] == -1 and math.isinf(delta[0]), (lam, delta)
        assert np.all(lam[1:] == 0) and np.all(delta[1:] == 0.0), (lam, delta)


def pin_line(variant=0):
    """Points 0..n-1 on a line, d_cut = 1: rho 2 at both ends, 3 inside; the
    highest point is id 1; lambda_i = i-1 for 2 <= i <= n-2, lambda_0 = 1,
    lambda_{n-1} = n-2; every delta is 1."""
    for n in (4, 9, 33):
        for dtype in (np.int32, np.float32):
            pts = W.line(n, dtype)
            rho = oracle.density(pts, 1.0, variant=variant)
            exp = np.full(n, 3)
            exp[0] = exp[-1] = 2
            assert np.array_equal(rho, exp), rho
            lam, delta = oracle.dependent(pts, rho, variant=variant)
            el = np.arange(n) - 1
            el[1] = -1
            el[0] = 1
            el[n - 1] = n - 2
            assert np.array_equal(lam, el), lam
            ed = np.ones(n)
            ed[1] = math.inf
            assert np.array_equal(delta, ed), delta


def pin_rho_vs_kdtree(variant=0):
    """rho against scipy's kd-tree ball count on integer points (exact
    distances); d_cut^2 is not an integer, so no rounding question arises,
    and d_cut = 5 exactly, where the inclusive boundary matters."""
    from scipy.spatial import cKDTree
    for seed, d in ((1, 2), (2, 3), (3, 5)):
        pts = W.random_blobs(600, d, seed, dtype=np.int32, scale=60.0, dup_frac=0.05)
        tree = cKDTree(pts.astype(np.float64))
        for dc in (4.7, 7.3):
            exp = tree.query_ball_point(pts.astype(np.float64), dc, return_length=True)
            rho = oracle.density(pts, dc, variant=variant)
            assert np.array_equal(rho, exp), (seed, dc)
        # integer radius: count |x - y|^2 <= 25 directly from integer offsets
        diff = pts[:, None, :].astype(np.int64) - pts[None, :, :].astype(np.int64)
        s = (diff * diff).sum(axis=2)
        exp = (s <= 25).sum(axis=1)
        rho = oracle.density(pts, 5.0, variant=variant)
        assert np.array_equal(rho, exp), seed


def pin_rho_parity_and_monotone(variant=0):
    """sum(rho) - n = 2 * #{pairs within d_cut} is even, and rho grows with d_cut."""
    pts = W.random_blobs(400, 3, 11, dtype=np.float32)
    prev = None
    for dc in (0.0, 0.01, 0.03, 0.07, 0.2):
        rho = oracle.density(pts, dc, variant=variant)
        assert (int(rho.sum()) - pts.shape[0]) % 2 == 0, dc
        if prev is not None:
            assert np.all(rho >= prev), dc
        prev = rho


def pin_zero_cut_prefix_nn(variant=0):
    """d_cut = 0 on distinct points: every rho is 1, so the order is the id
    order and lambda_i is the nearest neighbour among ids < i (smallest id on
    a distance tie), found here with scipy's kd-tree on each prefix."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(7)
    raw = rng.integers(0, 30, (600, 2))
    _, first = np.unique(raw, axis=0, return_index=True)
    pts = np.ascontiguousarray(raw[np.sort(first)][:250].astype(np.int32))
    n = pts.shape[0]
    rho = oracle.density(pts, 0.0, variant=variant)
    assert np.all(rho == 1)
    lam, delta = oracle.dependent(pts, rho, variant=variant)
    assert lam[0] == -1 and math.isinf(delta[0])
    x = pts.astype(np.float64)
    for i in range(1, n):
        tree = cKDTree(x[:i])
        dmin, _ = tree.query(x[i], k=1)
        near = tree.query_ball_point(x[i], dmin * (1 + 1e-9) + 1e-12)
        exact = [j for j in near if int(((pts[j].astype(np.int64) - pts[i]) ** 2).sum()) == int(round(dmin * dmin))]
        assert lam[i] == min(exact), (i, lam[i], exact)
        assert delta[i] == math.sqrt(float(((pts[lam[i]].astype(np.int64) - pts[i]) ** 2).sum()))


def pin_dependent_vs_sorted_prefix(variant=0):
    """Algorithm 2's reading: sort points by density, descending and stable
    (ties keep id order); the dependent point of the point at sorted position
    t is its nearest neighbour among positions < t, smallest id on a tie.
    Checked with scipy's kd-tree over each prefix, on integer points."""
    from scipy.spatial import cKDTree
    pts = W.random_blobs(300, 2, 5, dtype=np.int32, scale=40.0, dup_frac=0.05)
    rho = oracle.density(pts, 3.5, variant=0)
    lam, delta = oracle.dependent(pts, rho, variant=variant)
    order = np.argsort(-rho, kind="stable")
    x = pts.astype(np.float64)
    assert lam[order[0]] == -1 and math.isinf(delta[order[0]])
    for t in range(1, len(order)):
        i = order[t]
        prefix = order[:t]
        tree = cKDTree(x[prefix])
        dmin, _ = tree.query(x[i], k=1)
        near = tree.query_ball_point(x[i], dmin * (1 + 1e-9) + 1e-12)
        s_min = int(round(dmin * dmin))
        cands = [int(prefix[j]) for j in near
                 if int(((pts[prefix[j]].astype(np.int64) - pts[i]) ** 2).sum()) == s_min]
        assert lam[i] == min(cands), (i, lam[i], cands)
        assert delta[i] == math.sqrt(float(s_min))


def pin_labels_forest(variant=0):
    """Definitions 4-5 on c1-like data: noise iff rho < rho_noise; a center's
    label is itself; everyone else has its dependent point's label; the number
    of distinct labels equals the number of centers; lambda is strictly higher."""
    w = W.c1()
    pts = w.pts[:3000]
    rho = oracle.density(pts, w.d_cut[0], variant=variant)
    lam, delta = oracle.dependent(pts, rho, variant=variant)
    lab = oracle.cluster(rho, lam, delta, w.rho_noise[0], w.rho_min[0], w.delta_min[0], variant=variant)
    n = pts.shape[0]
    ids = np.arange(n)
    noise = rho < w.rho_noise[0]
    center = ~noise & ((lam < 0) | ((rho >= w.rho_min[0]) & (delta >= w.delta_min[0])))
    assert np.array_equal(lab == -1, noise)
    assert np.array_equal(lab[center], ids[center])
    rest = ~noise & ~center
    assert np.array_equal(lab[rest], lab[lam[rest]])
    assert len(set(lab[~noise].tolist())) == int(center.sum())
    roots = np.flatnonzero(lam < 0)
    assert len(roots) == 1
    r = roots[0]
    assert rho[r] == rho.max() and r == np.flatnonzero(rho == rho.max()).min()
    nr = lam >= 0
    hi = (rho[lam[nr]] > rho[nr]) | ((rho[lam[nr]] == rho[nr]) & (lam[nr] < ids[nr]))
    assert np.all(hi)


def pin_labels_split_thresholds(variant=0):
    """The hand-worked split-threshold example (tests/golden): a non-noise point
    with rho_noise <= rho < rho_min and delta >= delta_min is not a center
    (Definitions 4-5 read with two thresholds); with one threshold it is."""
    with open(os.path.join(GOLDEN, "labels_split_thresholds.json")) as f:
        g = json.load(f)
    base = np.array(g["points"], dtype=np.int64)
    for dtype, scale in ((np.int32, 1.0), (np.float32, 0.25)):
        pts = _as_dtype(base * scale, dtype)
        rho = oracle.density(pts, g["d_cut"] * scale, variant=variant)
        assert rho.tolist() == g["rho"]
        lam, delta = oracle.dependent(pts, rho, variant=variant)
        assert lam.tolist() == g["lambda"]
        assert np.array_equal(delta, _golden_delta(g["delta"]) * scale)
        lab = oracle.cluster(rho, lam, delta, g["rho_noise"], g["rho_min"], g["delta_min"] * scale,
                             variant=variant)
        assert lab.tolist() == g["label"]
        one = oracle.cluster(rho, lam, delta, g["rho_noise"], g["rho_noise"], g["delta_min"] * scale,
                             variant=variant)
        assert one.tolist() == g["label_single_threshold"]


ALL_PINS = [pin_hand_examples, pin_lattice_2d, pin_lattice_3d, pin_all_equal, pin_line,
            pin_rho_vs_kdtree, pin_rho_parity_and_monotone, pin_zero_cut_prefix_nn,
            pin_dependent_vs_sorted_prefix, pin_labels_forest, pin_labels_split_thresholds]
