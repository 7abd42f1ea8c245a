"""The float32 certification band, pinned on the CPU (no GPU).

The library filters distances in float32 and recounts in binary64 only the
pairs its band cannot decide (see dpc_cut_band in include/dpc.h).  The band
is what makes the float32 path exact, so it is checked here against the
binary64 truth on 1e7 seeded pairs drawn over the workloads' coordinate
ranges and d = 1..8, concentrated around the cutoff (where a wrong band would
show): the float32 value is evaluated exactly as the kernels evaluate it (t_k
rounded to float32, then a chain of fused multiply-adds in increasing k),
restated here with numpy float32/float64 arithmetic and an exact emulation of
fmaf; the truth is the canonical binary64 sum.  A band that ignores rounding
(t_in = t_out = fl32(d_cut^2)) is shown to fail on the same sample, so the
sample is sharp enough to catch a band that is too narrow.
"""
import math

import numpy as np
import pytest

import paper_2305_11335_gb300 as dpc
from paper_2305_11335_gb300 import _build

F32, F64 = np.float32, np.float64


@pytest.fixture(scope="module", autouse=True)
def lib():
    _build.build()
    return dpc.load()


def fmaf(a, b, c):
    """Correctly rounded float32 fma(a, b, c) of float32 arrays: a*b is exact
    in binary64 (24 + 24 bits), the sum's rounding error is recovered exactly
    with Knuth's two-sum, and the binary64 pair (hi, lo) is rounded once to
    float32 (lo only matters when hi sits exactly halfway between two
    float32 values)."""
    p = a.astype(F64) * b.astype(F64)
    cc = c.astype(F64)
    hi = p + cc
    bb = hi - p
    lo = (p - (hi - bb)) + (cc - bb)
    f = hi.astype(F32)
    toward = np.where(hi > f.astype(F64), np.inf, -np.inf).astype(F32)
    g = np.nextafter(f, toward)
    mid = (f.astype(F64) + g.astype(F64)) * 0.5
    at_mid = (hi == mid) & (f.astype(F64) != hi) & (lo != 0.0)
    # halfway: the exact value hi + lo lies on lo's side of the midpoint
    go_g = at_mid & (np.sign(lo) == np.sign(g.astype(F64) - f.astype(F64)))
    return np.where(go_g, g, f)


def test_fmaf_emulation_exact_cases():
    # exactly representable results
    a = np.array([1.5, 3.0, 0.0, 2.0 ** -10], F32)
    assert np.array_equal(fmaf(a, a, np.zeros(4, F32)), (a.astype(F64) ** 2).astype(F32))
    # a case that double rounding gets wrong: (1 + 2^-12)^2 + 2^-24 * 2^-1 ...
    t = F32(1.0 + 2.0 ** -12)
    exact = (1.0 + 2.0 ** -12) ** 2  # = 1 + 2^-11 + 2^-24, exact in binary64
    # add a tiny c that moves the exact sum just above the float32 midpoint
    c = F32(2.0 ** -60)
    want_up = np.nextafter(F32(exact), F32(2.0))  # the midpoint 1 + 2^-11 + 2^-24 rounds up only with c
    got = fmaf(np.array([t], F32), np.array([t], F32), np.array([c], F32))[0]
    assert got == want_up
    got0 = fmaf(np.array([t], F32), np.array([t], F32), np.array([0.0], F32))[0]
    assert got0 == F32(exact)  # ties to even without c


def s32_kernel(x, y):
    """The kernels' float32 value: t_k = fl32(x_k - y_k), s = fmaf(t_k, t_k, s)."""
    s = np.zeros(x.shape[0], F32)
    for k in range(x.shape[1]):
        t = (x[:, k] - y[:, k]).astype(F32)
        s = fmaf(t, t, s)
    return s


def s32_plain(x, y):
    """Another order the band must also cover: rounded square, then rounded add."""
    s = np.zeros(x.shape[0], F32)
    for k in range(x.shape[1]):
        t = (x[:, k] - y[:, k]).astype(F32)
        s = (s + (t * t).astype(F32)).astype(F32)
    return s


def s64_canonical(x, y):
    s = np.zeros(x.shape[0], F64)
    for k in range(x.shape[1]):
        t = x[:, k].astype(F64) - y[:, k].astype(F64)
        s = s + t * t
    return s


def sample_pairs(rng, m, d, extent, d_cut):
    """m pairs (a, b) in [0, extent]^d: most at distance d_cut (1 + eps) with
    |eps| in [1e-9, 1e-4], some exactly one cutoff apart along an axis, the
    rest anywhere up to three cutoffs."""
    a = (rng.random((m, d)) * extent).astype(F32)
    u = rng.normal(size=(m, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    kind = rng.random(m)
    eps = np.exp(rng.uniform(np.log(1e-9), np.log(1e-4), m)) * rng.choice([-1.0, 1.0], m)
    r = np.where(kind < 0.7, d_cut * (1.0 + eps), d_cut * rng.uniform(0.0, 3.0, m))
    b = (a.astype(F64) + u * r[:, None]).astype(F32)
    axis = kind > 0.9
    if axis.any():
        k = rng.integers(0, d, int(axis.sum()))
        bb = a[axis].copy()
        bb[np.arange(bb.shape[0]), k] = (bb[np.arange(bb.shape[0]), k].astype(F64) + d_cut).astype(F32)
        b[axis] = bb
    return a, b


# (extent, cutoff range) of the workloads: [0,1]^d mixtures (c2, c4, c5),
# the [0, 1e5]^3 seed spreader (c3), integer-valued coordinates up to 1e4 (c1)
RANGES = [(1.0, (1e-4, 0.2)), (1.0e5, (5.0, 300.0)), (1.0e4, (50.0, 1000.0)), (2.0 ** 20, (1.0, 4096.0))]


def test_band_decides_only_what_binary64_confirms():
    rng = np.random.default_rng(2024)
    chunks, per = 200, 50_000  # 1e7 pairs
    naive_wrong = 0
    ambiguous = 0
    boundary = 0
    for c in range(chunks):
        d = int(rng.integers(1, 9))
        extent, (lo, hi) = RANGES[c % len(RANGES)]
        d_cut = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if c % 7 == 0:
            d_cut = float(2.0 ** round(math.log2(d_cut)))  # exact sums exactly at the cutoff
        t_in, t_out, _, _ = dpc.cut_band(d_cut, d)
        dc2 = d_cut * d_cut
        a, b = sample_pairs(rng, per, d, extent, d_cut)
        s64 = s64_canonical(a, b)
        boundary += int((s64 == dc2).sum())
        for s32 in (s32_kernel(a, b), s32_plain(a, b)):
            inside = s32 <= F32(t_in)
            outside = s32 > F32(t_out)
            assert np.all(s64[inside] <= dc2), (c, d, d_cut)
            assert np.all(s64[outside] > dc2), (c, d, d_cut)
            ambiguous += int((~inside & ~outside).sum())
            naive = F32(dc2)
            naive_wrong += int(((s32 <= naive) & (s64 > dc2)).sum() + ((s32 > naive) & (s64 <= dc2)).sum())
    # the sample reaches the cutoff: exact boundary pairs exist, and a band
    # without a rounding allowance misclassifies some pairs
    assert boundary > 100
    assert naive_wrong > 100
    # the band is narrow: only pairs within ~1e-6 relative of the cutoff are left
    assert ambiguous < 0.2 * 2 * chunks * per


def test_band_ranks_dependent_candidates():
    """s32_b > s32_a * band_mul + band_add implies s64_b > s64_a (two pairs of
    one query with nearly equal distances)."""
    rng = np.random.default_rng(7)
    for c in range(60):
        d = int(rng.integers(1, 9))
        extent, (lo, hi) = RANGES[c % len(RANGES)]
        d_cut = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        _, _, mul, add = dpc.cut_band(d_cut, d)
        m = 50_000
        q = (rng.random((m, d)) * extent).astype(F32)
        u1 = rng.normal(size=(m, d))
        u1 /= np.linalg.norm(u1, axis=1, keepdims=True)
        u2 = rng.normal(size=(m, d))
        u2 /= np.linalg.norm(u2, axis=1, keepdims=True)
        r1 = d_cut * rng.uniform(0.01, 5.0, m)
        r2 = r1 * (1.0 + np.exp(rng.uniform(np.log(1e-9), np.log(1e-5), m)) * rng.choice([-1.0, 1.0], m))
        a = (q.astype(F64) + u1 * r1[:, None]).astype(F32)
        b = (q.astype(F64) + u2 * r2[:, None]).astype(F32)
        sa, sb = s32_kernel(q, a), s32_kernel(q, b)
        ta, tb = s64_canonical(q, a), s64_canonical(q, b)
        sure = sb > sa * F32(mul) + F32(add)
        assert np.all(tb[sure] > ta[sure]), (c, d)
        sure = sa > sb * F32(mul) + F32(add)
        assert np.all(ta[sure] > tb[sure]), (c, d)


def test_cut_band_rejects_bad_arguments():
    for dc, dim in ((1.0, 0), (1.0, 9), (-1.0, 2), (math.nan, 2), (math.inf, 3)):
        with pytest.raises(dpc.DpcError):
            dpc.cut_band(dc, dim)
