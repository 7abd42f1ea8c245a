"""The kd-tree oracle (oracle/dpc_oracle_tree.c) against the brute-force one.

The kd-tree oracle is what the full-size GPU parity tests compare with; it
must give exactly what the O(n^2) definitions give (Definitions 1-3 under the
oracle's fixed readings), which are themselves pinned in test_oracle.py.
Seeded fuzz cases cover d in {1, 2, 3, 5, 7, 8}, int32 and float32 points,
exact duplicates, lattices whose spacing equals the cutoff (many distances
exactly at d_cut and many exact distance ties), several cutoffs per call in
any order, the noise skip, and the batched form.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def brute(pts, d_cuts, rho_skip=0):
    rows = {"rho": [], "lam": [], "delta": []}
    for dc in d_cuts:
        rho = oracle.density(pts, dc)
        lam, delta = oracle.dependent(pts, rho, rho_skip=rho_skip)
        rows["rho"].append(rho)
        rows["lam"].append(lam)
        rows["delta"].append(delta)
    return {k: np.stack(v) for k, v in rows.items()}


def assert_equal_runs(got, want, what):
    assert np.array_equal(got["rho"], want["rho"]), what + " rho"
    assert np.array_equal(got["lam"], want["lam"]), what + " lambda"
    assert np.array_equal(got["delta"].view(np.int64), want["delta"].view(np.int64)), what + " delta"


def fuzz_case(k):
    """Case k of the seeded fuzz set: (points, cutoffs, description)."""
    rng = np.random.default_rng(1000 + k)
    kind = k % 5
    d = [1, 2, 3, 5, 7, 8][int(rng.integers(0, 6))]
    n = int(np.exp(rng.uniform(np.log(2), np.log(2500))))
    if kind == 0:   # float blobs + noise, duplicates
        pts = W.random_blobs(n, d, 5000 + k, dtype=np.float32, dup_frac=0.05)
        base = 0.05 * math.sqrt(d)
    elif kind == 1:  # int blobs (exact integer distances, many ties)
        pts = W.random_blobs(n, d, 5000 + k, dtype=np.int32, scale=60.0, dup_frac=0.05)
        base = 3.0 * math.sqrt(d)
    elif kind == 2:  # lattice, cutoff at exactly the spacing (or a diagonal)
        side = max(2, int(round(n ** (1.0 / min(d, 3)))))
        dd = min(d, 3)
        spacing = int(rng.integers(1, 4))
        pts = W.lattice(side, dd, spacing)
        if rng.random() < 0.5:
            pts = pts.astype(np.float32) * np.float32(0.25)  # exact in binary32
            spacing = spacing * 0.25
        perm = rng.permutation(pts.shape[0])
        pts = np.ascontiguousarray(pts[perm])
        base = float(spacing)
        return pts, [base, base * math.sqrt(2.0), base * 2.0][: 1 + int(rng.integers(0, 3))], \
            "lattice d=%d side=%d spacing=%g %s" % (dd, side, spacing, pts.dtype)
    elif kind == 3:  # tiny sets, all-equal and near-equal points
        n = int(rng.integers(1, 40))
        pts = np.repeat(rng.random((max(1, n // 4), d)).astype(np.float32), 4, axis=0)[:n]
        pts = np.ascontiguousarray(pts)
        base = 0.3
    else:            # wide extent, tight clusters
        pts = W.wide_clusters(n, d, 5000 + k, extent=1.0e5, sigma=3.0, n_centers=8)
        base = 6.0
    ncut = int(rng.integers(1, 4))
    cuts = [base * f for f in rng.permutation([0.5, 1.0, 1.7])[:ncut]]
    if rng.random() < 0.1:
        cuts[0] = 0.0
    return pts, cuts, "kind %d n=%d d=%d %s" % (kind, pts.shape[0], d, pts.dtype)


@pytest.mark.parametrize("k", range(200))
def test_tree_equals_brute_force(k):
    pts, cuts, what = fuzz_case(k)
    got = oracle.tree_run(pts, cuts)
    assert_equal_runs(got, brute(pts, cuts), what)


@pytest.mark.parametrize("dtype,d", [(np.float32, 2), (np.int32, 3), (np.float32, 5), (np.float32, 7)])
def test_tree_equals_brute_force_20k(dtype, d):
    """The largest fuzz size, n = 2e4."""
    scale = 400.0 if dtype == np.int32 else 1.0
    pts = W.random_blobs(20000, d, 77 + d, dtype=dtype, scale=scale, dup_frac=0.01)
    cuts = [0.02 * scale * math.sqrt(d), 0.05 * scale * math.sqrt(d)]
    assert_equal_runs(oracle.tree_run(pts, cuts), brute(pts, cuts), "n=2e4 d=%d" % d)


def test_tree_noise_skip():
    pts = W.random_blobs(3000, 3, 9, dup_frac=0.02)
    cuts = [0.03, 0.06]
    got = oracle.tree_run(pts, cuts, rho_skip=4)
    assert_equal_runs(got, brute(pts, cuts, rho_skip=4), "skip")
    assert np.isnan(got["delta"][0]).any()


def test_tree_density_only_and_degenerate():
    one = np.zeros((1, 3), np.float32)
    r = oracle.tree_run(one, [1.0])
    assert r["rho"].tolist() == [[1]] and r["lam"].tolist() == [[-1]] and math.isinf(r["delta"][0, 0])
    r = oracle.tree_run(np.zeros((0, 2), np.float32), [1.0])
    assert r["rho"].shape == (1, 0)
    pts = W.random_blobs(500, 2, 3)
    r = oracle.tree_run(pts, [0.05], dependent=False)
    assert r["lam"] is None and np.array_equal(r["rho"][0], oracle.density(pts, 0.05))


def test_tree_batch_equals_single_sets():
    """The batched form (one thread per instance) gives each instance what the
    single-set form gives, with instance-local ids."""
    rng = np.random.default_rng(5)
    sets, cuts = [], []
    for i in range(12):
        d = [2, 3, 5][i % 3]
        n = int(rng.integers(0, 1500))
        sets.append(W.random_blobs(n, d, 300 + i, dup_frac=0.03) if n else np.zeros((0, d), np.float32))
        c0 = 0.03 * math.sqrt(d)
        cuts.append([c0, c0 * 1.25, c0 * 1.5625])
    flat = np.concatenate([s.ravel() for s in sets]).astype(np.float32)
    po = np.concatenate([[0], np.cumsum([s.shape[0] for s in sets])])
    co = np.concatenate([[0], np.cumsum([s.size for s in sets])[:-1]])
    dims = [s.shape[1] for s in sets]
    got = oracle.tree_batch(flat, po, co, dims, cuts)
    for i, s in enumerate(sets):
        want = oracle.tree_run(s, cuts[i])
        part = {k: v[:, po[i]:po[i + 1]] for k, v in got.items()}
        assert_equal_runs(part, want, "instance %d" % i)
