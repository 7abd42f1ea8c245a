"""The CPU oracle against its pins (no GPU).

Each pin in ``_pins.py`` checks the oracle against a hand-worked example, a
closed form, an invariant, or a library routine (scipy's kd-tree), never
against itself.  The planted-mistake tests show every deviation the oracle can
be switched into is caught by at least one pin.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _pins import ALL_PINS

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_pin_holds(pin):
    pin(0)


PLANTED = [oracle.VAR_EXCLUSIVE, oracle.VAR_NO_SELF, oracle.VAR_TIE_LARGER_ID,
           oracle.VAR_DIST_TIE_LARGER, oracle.VAR_DROP_LAST_DIM, oracle.VAR_CENTER_NO_RHO_MIN]


def test_center_threshold_mistake_caught_by_hand_example():
    """Dropping rho >= rho_min from the center rule is caught by the
    hand-worked split-threshold example itself, not only by a restatement."""
    from _pins import pin_labels_split_thresholds
    pin_labels_split_thresholds(0)
    with pytest.raises(AssertionError):
        pin_labels_split_thresholds(oracle.VAR_CENTER_NO_RHO_MIN)


@pytest.mark.parametrize("variant", PLANTED)
def test_planted_mistake_is_caught(variant):
    failed = []
    for pin in ALL_PINS:
        try:
            pin(variant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "no pin catches oracle variant %d" % variant


def test_sqrt_reading_differs_only_at_rounding():
    """The alternative reading sqrt(s) <= d_cut agrees with s <= d_cut^2 on
    exact lattice distances; it is kept only to count the two readings apart."""
    pts = W.lattice(6, 2, 1)
    for dc in (1.0, 2.0, math.sqrt(2.0), 2.5):
        a = oracle.density(pts, dc)
        b = oracle.density(pts, dc, variant=oracle.VAR_SQRT_COMPARE)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype,d,seed", [(np.int32, 2, 1), (np.float32, 2, 2), (np.float32, 3, 3),
                                          (np.float32, 5, 4), (np.int32, 8, 5), (np.float32, 1, 6)])
def test_sampled_dependent_equals_full(dtype, d, seed):
    """The on-demand form (walk points in distance order, compute each density
    from scratch) agrees with the full form (density array, key-filtered scan)."""
    scale = 50.0 if dtype == np.int32 else 1.0
    pts = W.random_blobs(500, d, seed, dtype=dtype, scale=scale, dup_frac=0.05)
    dc = 0.08 * scale * math.sqrt(d)
    rho = oracle.density(pts, dc)
    lam, delta = oracle.dependent(pts, rho)
    idx = np.arange(0, 500, 7)
    l2, d2, r2, ok = oracle.dependent_at(pts, dc, idx, max_checks=500)
    assert ok.all()
    assert np.array_equal(r2, rho[idx])
    assert np.array_equal(l2, lam[idx])
    assert np.array_equal(d2, delta[idx])


def test_sampled_dependent_reports_unresolved():
    pts = W.line(50, np.int32)
    # the highest point needs every other point examined
    lam, delta, rho, ok = oracle.dependent_at(pts, 1.0, np.array([1, 2]), max_checks=3)
    assert not ok[0] and ok[1] and lam[1] == 1


def test_rho_skip():
    pts = W.random_blobs(200, 2, 9)
    rho = oracle.density(pts, 0.05)
    lam, delta = oracle.dependent(pts, rho, rho_skip=3)
    skip = rho < 3
    assert np.all(lam[skip] == -1) and np.all(np.isnan(delta[skip]))
    lam0, delta0 = oracle.dependent(pts, rho)
    assert np.array_equal(lam[~skip], lam0[~skip])


def test_kth_sqdist_matches_sorting():
    pts = W.random_blobs(300, 3, 12)
    x = pts.astype(np.float64)
    idx = np.array([0, 5, 77, 299])
    for k in (1, 2, 30):
        got = oracle.kth_sqdist(pts, idx, k)
        for t, i in enumerate(idx):
            diff = x - x[i]
            s = np.sort((diff * diff).sum(axis=1))
            assert got[t] == pytest.approx(s[k - 1], rel=1e-12, abs=0)


def test_cluster_rejects_cycles():
    rho = np.array([5, 5, 5], np.int32)
    lam = np.array([1, 2, 0], np.int32)
    delta = np.array([1.0, 1.0, 1.0])
    with pytest.raises(RuntimeError):
        oracle.cluster(rho, lam, delta, 1, 1, 10.0)


def test_empty_and_single():
    e = np.zeros((0, 2), np.float32)
    r = oracle.run(e, 1.0, 1, 1, 1.0)
    assert all(v.shape == (0,) for v in r.values())
    one = np.array([[1.5, 2.0]], np.float32)
    r = oracle.run(one, 1.0, 1, 1, 1.0)
    assert r["rho"].tolist() == [1] and r["lam"].tolist() == [-1]
    assert math.isinf(r["delta"][0]) and r["label"].tolist() == [0]
