"""Pins for the decision-graph oracle (no GPU).

Each pin checks ``oracle.decision_graph`` against a hand-worked example, an
exact product computed with rationals, or an order/bin property checked point
by point; the planted-mistake test shows every deviation the oracle can be
switched into fails at least one pin.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

INF = math.inf
NAN = math.nan


def _hand(variant):
    # gamma = [inf, 1.5, 4, 4, NaN, 0]: the top point first, the tie at 4 by
    # the smaller id, the skipped point (NaN delta) left out
    rho = [3, 1, 2, 2, 5, 1]
    delta = [INF, 1.5, 2.0, 2.0, NAN, 0.0]
    out = oracle.decision_graph(rho, delta, 7, 3, 4, 1.0, variant=variant)
    assert out["top"].tolist() == [0, 2, 3, 1, 5, -1, -1]
    g = out["gamma"]
    assert g[0] == INF and g[1] == 4.0 and g[2] == 4.0 and g[3] == 1.5 and g[4] == 0.0
    assert math.isnan(g[5]) and math.isnan(g[6])
    # rho bins floor(log2 rho) -> [1, 0, 1, 1, -, 0]; delta bins with lo = 1:
    # inf -> last (3), 1.5 -> 0, 2 -> 1, 2 -> 1, 0 -> 0
    want = np.zeros((3, 4), dtype=np.int64)
    want[1, 3] += 1
    want[0, 0] += 1
    want[1, 1] += 2
    want[0, 0] += 1
    assert (out["hist"] == want).all(), out["hist"]


def _hand_k2(variant):
    out = oracle.decision_graph([3, 1, 2, 2], [INF, 1.5, 2.0, 2.0], 2, variant=variant)
    assert out["top"].tolist() == [0, 2]


def _exact_products(variant):
    rng = np.random.default_rng(5)
    rho = rng.integers(1, 1 << 30, 200).astype(np.int32)
    delta = rng.random(200) * 10.0 ** rng.integers(-8, 8, 200)
    out = oracle.decision_graph(rho, delta, 200, variant=variant)
    for j, i in enumerate(out["top"]):
        want = float(Fraction(int(rho[i])) * Fraction(float(delta[i])))  # correctly rounded
        assert out["gamma"][j] == want


def _order_property(variant):
    # selected rows are exactly the k best (score, -id) pairs: no left-out point
    # beats the last selected one, and the rows are in order
    rng = np.random.default_rng(9)
    rho = rng.integers(1, 5, 300).astype(np.int32)
    delta = rng.integers(0, 4, 300).astype(np.float64)  # many exact ties
    delta[rng.integers(0, 300, 20)] = NAN
    delta[7] = INF
    k = 40
    out = oracle.decision_graph(rho, delta, k, variant=variant)
    top, gam = out["top"], out["gamma"]
    chosen = set(top.tolist())
    for j in range(k - 1):
        a, b = (gam[j], -top[j]), (gam[j + 1], -top[j + 1])
        assert a > b
    last = (gam[k - 1], -top[k - 1])
    for i in range(300):
        if i in chosen or math.isnan(delta[i]):
            continue
        assert (float(rho[i]) * delta[i], -i) < last
    assert top[0] == 7 and gam[0] == INF


def _bin_property(variant):
    rng = np.random.default_rng(11)
    n = 500
    rho = rng.integers(1, 1 << 20, n).astype(np.int32)
    lo = 1e-3
    delta = lo * 2.0 ** rng.uniform(-3, 30, n)
    delta[:5] = [lo, lo * 2, lo * 4, INF, lo / 2]
    delta[5] = NAN
    out = oracle.decision_graph(rho, delta, 0, 21, 24, lo, variant=variant)
    h = out["hist"]
    assert h.sum() == n - 1
    want = np.zeros_like(h)
    for i in range(n):
        if math.isnan(delta[i]):
            continue
        r = int(rho[i])
        a = 0
        while a + 1 < 21 and (1 << (a + 1)) <= r:
            a += 1
        if not delta[i] > lo:
            b = 0
        elif math.isinf(delta[i]):
            b = 23
        else:
            q = delta[i] / lo
            b = 0
            while b + 1 < 24 and math.ldexp(1.0, b + 1) <= q:
                b += 1
        want[a, b] += 1
    assert (h == want).all()


PINS = [_hand, _hand_k2, _exact_products, _order_property, _bin_property]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_decision_pin_holds(pin):
    pin(0)


@pytest.mark.parametrize("variant", [oracle.DG_TIE_LARGER_ID, oracle.DG_DROP_INF, oracle.DG_DELTA_BIN_UP,
                                     oracle.DG_SUM_NOT_PRODUCT])
def test_decision_planted_mistake_is_caught(variant):
    failed = []
    for pin in PINS:
        try:
            pin(variant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "no pin catches decision-graph variant %d" % variant


def test_decision_empty_and_short_rows():
    out = oracle.decision_graph([], [], 3, 2, 2, 1.0)
    assert out["top"].tolist() == [-1, -1, -1] and out["hist"].sum() == 0
    out = oracle.decision_graph([1, 1], [NAN, NAN], 2)
    assert out["top"].tolist() == [-1, -1]
