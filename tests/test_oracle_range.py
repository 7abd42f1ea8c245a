"""Pins for the priority range search oracle (no GPU).

``oracle.priority_range`` is checked against a hand-worked example, exact
boundary cases, a partition identity (two boxes split at a value between
coordinates count every point once) and monotonicity in the threshold; the
planted-mistake test shows every deviation the oracle can be switched into
fails at least one pin.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _hand(variant):
    # points on a 3x3 integer grid, densities chosen by hand
    pts = np.array([[x, y] for y in range(3) for x in range(3)], dtype=np.int32)  # id = 3y + x
    rho = np.array([5, 1, 7, 2, 9, 3, 4, 8, 6], dtype=np.int32)
    # box [0,1] x [0,1] holds ids 0, 1, 3, 4 (the corners are on its boundary)
    got = oracle.priority_range(pts, rho, [0, 0], [1, 1], 2, variant=variant)
    assert got.tolist() == [0, 4]          # rho 5, 9 exceed 2; id 3 has rho exactly 2
    got = oracle.priority_range(pts, rho, [0.5, 0.5], [2, 2], 0, variant=variant)
    assert got.tolist() == [4, 5, 7, 8]


def _boundary(variant):
    pts = np.array([[1.5, -2.0, 0.25], [1.5, -2.0, 0.5], [3.0, 0.0, 0.0]], dtype=np.float32)
    rho = np.array([3, 3, 3], dtype=np.int32)
    # a degenerate box holding exactly point 0
    got = oracle.priority_range(pts, rho, [1.5, -2.0, 0.25], [1.5, -2.0, 0.25], 2, variant=variant)
    assert got.tolist() == [0]
    # the last coordinate alone separates points 0 and 1
    got = oracle.priority_range(pts, rho, [1.5, -2.0, 0.3], [1.5, -2.0, 1.0], 2, variant=variant)
    assert got.tolist() == [1]


def _partition(variant):
    rng = np.random.default_rng(3)
    pts = W.random_blobs(3000, 3, 17)
    rho = rng.integers(0, 50, 3000).astype(np.int32)
    lo, hi = np.array([0.1, 0.2, 0.0]), np.array([0.9, 0.7, 0.8])
    whole = oracle.priority_range(pts, rho, lo, hi, 20, variant=variant)
    # split the first axis at a value no coordinate takes (float32 points, a
    # float64 split value strictly between two float32 numbers)
    xs = np.unique(pts[:, 0].astype(np.float64))
    i = np.searchsorted(xs, 0.5)
    m = 0.5 * (xs[i - 1] + xs[i])
    assert m not in set(xs.tolist())
    a = oracle.priority_range(pts, rho, lo, [m, hi[1], hi[2]], 20, variant=variant)
    b = oracle.priority_range(pts, rho, [m, lo[1], lo[2]], hi, 20, variant=variant)
    assert sorted(a.tolist() + b.tolist()) == whole.tolist()
    # brute force on a few points, one by one
    for j in range(0, 3000, 97):
        inside = all(lo[k] <= float(pts[j, k]) <= hi[k] for k in range(3)) and rho[j] > 20
        assert (j in set(whole.tolist())) == inside


def _monotone(variant):
    rng = np.random.default_rng(4)
    pts = rng.integers(-50, 50, (2000, 2)).astype(np.int32)
    rho = rng.integers(1, 10, 2000).astype(np.int32)
    prev = None
    for q in range(10, -1, -1):
        cur = set(oracle.priority_range(pts, rho, [-10, -20], [10, 5], q, variant=variant).tolist())
        if prev is not None:
            assert prev <= cur
            assert cur - prev == {i for i in cur if rho[i] == q + 1}
        prev = cur
    # threshold below every density and a box around everything: every point
    assert len(oracle.priority_range(pts, rho, [-50, -50], [49, 49], 0, variant=variant)) == 2000


PINS = [_hand, _boundary, _partition, _monotone]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_range_pin_holds(pin):
    pin(0)


@pytest.mark.parametrize("variant", [oracle.PR_GE, oracle.PR_OPEN_BOX, oracle.PR_DROP_LAST])
def test_range_planted_mistake_is_caught(variant):
    failed = []
    for pin in PINS:
        try:
            pin(variant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "no pin catches priority-range variant %d" % variant
