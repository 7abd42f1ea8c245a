"""Seeded synthetic point sets for exact Density Peaks Clustering.

This module only draws random points: it holds none of the clustering
arithmetic (no distances, densities or dependent points), so the CUDA path and
the CPU oracle can both be fed from it.  Parameters that depend on the data
(a ``d_cut`` giving a target median density, the noise threshold) are read from
``tests/golden/workload_params.json``, which a committed script computes with
the oracle alone.

The paper evaluates on uniform, simden and varden 2-D sets with n up to 1e7
(Section 7, Table 2) and on real data sets that are not available here; the
generators below stand in for them:

* ``c1``  n=1e4, d=2, int32: 5 isotropic Gaussian blobs + 10% uniform noise.
* ``c2``  n=1e6, d=2, float32: 50-blob Gaussian mixture + 5% uniform noise.
* ``c3``  n=1e7, d=3, float32: a seed-spreader random walk (the random-walk
          style of simden/varden) + 0.1% uniform noise.
* ``c4``  4096 independent float32 instances, n log-uniform in [1e3, 2e5],
          d in {2, 3, 5}, each a 2-40 blob mixture, 8 d_cut values each.
* ``c5``  n=2e6, d=7, float32: 30 anisotropic Gaussian blobs + 2% noise,
          4 d_cut values.

All use numpy's PCG64 through ``np.random.default_rng(seed)``; every point set
is shuffled once so that point ids carry no spatial order.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

_PARAMS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                            "workload_params.json")
_C4_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "c4_params.json")


@dataclass
class Workload:
    name: str
    pts: np.ndarray                 # (n, d) int32 or float32, C-contiguous
    d_cut: list                     # one or more cutoffs (a sweep)
    rho_noise: list                 # per d_cut
    rho_min: list                   # per d_cut
    delta_min: list                 # per d_cut
    noise_ids: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def d(self) -> int:
        return int(self.pts.shape[1])


def load_params() -> dict:
    if not os.path.exists(_PARAMS_PATH):
        return {}
    with open(_PARAMS_PATH) as f:
        return json.load(f)


def _shuffle(rng, pts, n_noise_tail):
    """Shuffle rows; return (shuffled points, ids of the rows that were the
    last ``n_noise_tail`` rows before shuffling)."""
    n = pts.shape[0]
    perm = rng.permutation(n)
    out = np.ascontiguousarray(pts[perm])
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n, dtype=np.int64)
    noise_ids = np.sort(inv[n - n_noise_tail:]) if n_noise_tail else np.zeros(0, np.int64)
    return out, noise_ids


def gaussian_mixture(rng, n_blob_pts, n_blobs, d, sigma_lo, sigma_hi, weights=None):
    """Isotropic Gaussian blobs, centers U[0,1)^d, sigma log-uniform."""
    if weights is None:
        weights = rng.dirichlet(np.ones(n_blobs))
    counts = rng.multinomial(n_blob_pts, weights)
    centers = rng.random((n_blobs, d))
    sigma = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_blobs))
    parts = [centers[b] + sigma[b] * rng.standard_normal((counts[b], d)) for b in range(n_blobs)]
    return np.concatenate(parts, axis=0) if parts else np.zeros((0, d))


# ---------------------------------------------------------------------------
# the five workload families


def c1(seed: int = 0) -> Workload:
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, 1e4, (5, 2))
    sigma = rng.uniform(100.0, 400.0, 5)
    blobs = np.concatenate([centers[b] + sigma[b] * rng.standard_normal((1800, 2)) for b in range(5)])
    noise = rng.uniform(0.0, 1e4, (1000, 2))
    pts = np.concatenate([blobs, noise])
    pts, noise_ids = _shuffle(rng, pts, 1000)
    pts = np.rint(pts).astype(np.int32)
    return Workload("c1_blobs_int32_n1e4_d2", pts, [150.0], [3], [10], [1000.0], noise_ids)


def c2_points(seed: int = 2) -> tuple:
    rng = np.random.default_rng(seed)
    blobs = gaussian_mixture(rng, 950_000, 50, 2, 1e-3, 2e-2)
    noise = rng.random((50_000, 2))
    pts, noise_ids = _shuffle(rng, np.concatenate([blobs, noise]), 50_000)
    return pts.astype(np.float32), noise_ids


def c2(seed: int = 2) -> Workload:
    pts, noise_ids = c2_points(seed)
    p = load_params().get("c2", {})
    dc = p.get("d_cut", float("nan"))
    rmin = p.get("rho_min", 0)
    return Workload("c2_mixture_f32_n1e6_d2", pts, [dc], [rmin], [rmin], [0.05], noise_ids)


def c3_points(seed: int = 3, steps: int = 99_900, per_step: int = 100, n_noise: int = 10_000,
              box: float = 1e5, step_len: float = 50.0, radius: float = 100.0,
              restart_p: float = 1e-4, d: int = 3) -> tuple:
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((steps, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    restart = rng.random(steps) < restart_p
    restart_pos = rng.uniform(0.0, box, (steps, d))
    pos = rng.uniform(0.0, box, d).tolist()
    centers = np.empty((steps, d))
    dl = dirs.tolist()
    rl = restart.tolist()
    rp = restart_pos.tolist()
    for t in range(steps):
        dx = dl[t]
        pos = [min(max(pos[k] + step_len * dx[k], 0.0), box) for k in range(d)]
        centers[t] = pos
        if rl[t]:
            pos = rp[t]
    # per_step points uniform in the ball of `radius` around each walk position
    m = steps * per_step
    u = rng.standard_normal((m, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = rng.random(m)
    r = radius * (np.cbrt(v) if d == 3 else v ** (1.0 / d))
    cloud = np.repeat(centers, per_step, axis=0) + u * r[:, None]
    del u, r
    noise = rng.uniform(0.0, box, (n_noise, d))
    pts, noise_ids = _shuffle(rng, np.concatenate([cloud, noise]), n_noise)
    return pts.astype(np.float32), noise_ids


def c3(seed: int = 3) -> Workload:
    pts, noise_ids = c3_points(seed)
    p = load_params().get("c3", {})
    rmin = p.get("rho_min", 0)
    return Workload("c3_seedspreader_f32_n1e7_d3", pts, [30.0], [rmin], [rmin], [1000.0], noise_ids)


def spreader(n: int, d: int, seed: int = 3) -> Workload:
    """The seed-spreader family at any size: the walk of ``c3_points`` in d
    dimensions with 100 points per step and about 0.1% uniform noise in the
    [0, 1e5]^d box, with the paper's synthetic hyper-parameters (d_cut = 30,
    rho_min = 0, delta_min = 100).  n = 1e7, d = 3 is exactly ``c3``'s point
    set; d = 2 stands in for simden."""
    steps = max(1, int(round(0.999 * n / 100)))
    n_noise = max(0, n - 100 * steps)
    pts, noise_ids = c3_points(seed, steps=steps, per_step=100, n_noise=n_noise, d=d)
    pts = pts[:n] if pts.shape[0] > n else pts
    return Workload("spreader_f32_n%d_d%d" % (n, d), np.ascontiguousarray(pts), [30.0], [0], [0], [100.0],
                    noise_ids[noise_ids < n])


def c5_points(seed: int = 5, n_blob_pts: int = 1_960_000, n_blobs: int = 30, n_noise: int = 40_000,
              d: int = 7) -> tuple:
    rng = np.random.default_rng(seed)
    counts = np.full(n_blobs, n_blob_pts // n_blobs)
    counts[: n_blob_pts % n_blobs] += 1
    centers = rng.random((n_blobs, d))
    parts = []
    for b in range(n_blobs):
        q, r = np.linalg.qr(rng.standard_normal((d, d)))
        q = q * np.sign(np.diag(r))[None, :]
        lam = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), d))
        z = rng.standard_normal((counts[b], d)) * np.sqrt(lam)[None, :]
        parts.append(centers[b] + z @ q.T)
    noise = rng.random((n_noise, d))
    pts, noise_ids = _shuffle(rng, np.concatenate(parts + [noise]), n_noise)
    return pts.astype(np.float32), noise_ids


def c5(seed: int = 5) -> Workload:
    pts, noise_ids = c5_points(seed)
    p = load_params().get("c5", {})
    dc0 = p.get("d_cut0", float("nan"))
    cuts = [dc0 * 1.25 ** k for k in range(4)]
    rmins = p.get("rho_min", [0] * 4)
    return Workload("c5_aniso_f32_n2e6_d7", pts, cuts, list(rmins), list(rmins),
                    [10.0 * dc0] * 4, noise_ids)


def c4_instance_specs(seed: int = 4, n_inst: int = 4096):
    """(n_i, d_i, n_blobs_i, child seed) for every batched instance."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(math.log(1e3), math.log(2e5), n_inst))).astype(np.int64)
    d = rng.choice(np.array([2, 3, 5]), n_inst)
    blobs = rng.integers(2, 41, n_inst)
    child = np.random.SeedSequence(seed).spawn(n_inst)
    return [(int(n[i]), int(d[i]), int(blobs[i]), child[i]) for i in range(n_inst)]


def c4_instance(spec) -> np.ndarray:
    n, d, nb, ss = spec
    rng = np.random.default_rng(ss)
    pts = gaussian_mixture(rng, n, nb, d, 1e-3, 2e-2)
    pts, _ = _shuffle(rng, pts, 0)
    return pts.astype(np.float32)


C4_NCUT = 8


@dataclass
class BatchWorkload:
    """Independent instances packed back to back (instance i owns rows
    [offset[i], offset[i+1]) of ``flat`` viewed per instance as (n_i, d_i))."""
    name: str
    sizes: list
    dims: list
    flat: np.ndarray                # float32, every instance's coordinates concatenated
    coord_offset: list              # element offset of each instance in ``flat``
    d_cut: list                     # [n_inst][n_dcut]
    rho_noise: list                 # [n_inst * n_dcut]
    rho_min: list                   # [n_inst * n_dcut]
    delta_min: list                 # [n_inst * n_dcut]

    @property
    def n_inst(self) -> int:
        return len(self.sizes)

    @property
    def N(self) -> int:
        return int(sum(self.sizes))

    def instance(self, i: int) -> np.ndarray:
        o = self.coord_offset[i]
        return self.flat[o:o + self.sizes[i] * self.dims[i]].reshape(self.sizes[i], self.dims[i])


def c4(seed: int = 4, n_inst: int = 4096) -> BatchWorkload:
    """The batched workload: per instance the sweep d_cut0 * 1.25^k (k < 8),
    rho_noise = rho_min = 2 x median density at each cutoff, delta_min =
    5 d_cut (d_cut0 and the densities from tests/golden/c4_params.json)."""
    specs = c4_instance_specs(seed, n_inst)
    with open(_C4_PATH) as f:
        par = json.load(f)
    parts, co, o = [], [], 0
    for s in specs:
        p = c4_instance(s)
        parts.append(p.reshape(-1))
        co.append(o)
        o += p.size
    flat = np.concatenate(parts)
    cuts = [[par["d_cut0"][i] * 1.25 ** k for k in range(C4_NCUT)] for i in range(n_inst)]
    rmin = [int(r) for i in range(n_inst) for r in par["rho_min"][i]]
    dmin = [5.0 * c for row in cuts for c in row]
    return BatchWorkload("c4_batch4096_f32_d235_x8cuts", [s[0] for s in specs], [s[1] for s in specs],
                         flat, co, cuts, list(rmin), rmin, dmin)


# ---------------------------------------------------------------------------
# small structured sets for tests


def lattice(k: int, dim: int = 2, spacing: int = 1, dtype=np.int32) -> np.ndarray:
    """The k^dim integer lattice with the given spacing, row-major ids."""
    axes = [np.arange(k) * spacing] * dim
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    return np.ascontiguousarray(g.astype(dtype))


def line(n: int, dtype=np.int32) -> np.ndarray:
    """Points 0, 1, ..., n-1 on a line, id i at coordinate i."""
    return np.arange(n, dtype=dtype).reshape(n, 1).copy()


def all_equal(n: int, d: int, value=3.0, dtype=np.float32) -> np.ndarray:
    return np.full((n, d), value, dtype=dtype)


def random_blobs(n: int, d: int, seed: int, dtype=np.float32, n_blobs: int = 4, scale: float = 1.0,
                 dup_frac: float = 0.0, noise_frac: float = 0.1) -> np.ndarray:
    """A small Gaussian mixture with uniform noise and optional exact duplicates."""
    rng = np.random.default_rng(seed)
    nn = int(round(n * noise_frac))
    blobs = gaussian_mixture(rng, n - nn, n_blobs, d, 0.02, 0.1)
    noise = rng.random((nn, d))
    pts = np.concatenate([blobs, noise]) * scale
    ndup = int(round(n * dup_frac))
    if ndup and n > 1:
        src = rng.integers(0, n, ndup)
        dst = rng.integers(0, n, ndup)
        pts[dst] = pts[src]
    pts, _ = _shuffle(rng, pts, 0)
    if np.issubdtype(np.dtype(dtype), np.integer):
        return np.rint(pts).astype(dtype)
    return pts.astype(dtype)


def wide_clusters(n: int, d: int, seed: int, extent: float = 2.0e6, sigma: float = 20.0,
                  n_centers: int = 64, dtype=np.int32) -> np.ndarray:
    """Tight isotropic clusters (sigma) around n_centers centers drawn
    uniformly in [0, extent)^d: a bounding box many thousand cutoffs wide with
    non-trivial densities inside the clusters."""
    rng = np.random.default_rng(seed)
    centers = rng.random((n_centers, d)) * extent
    which = rng.integers(0, n_centers, n)
    pts = centers[which] + rng.normal(0.0, sigma, (n, d))
    pts, _ = _shuffle(rng, pts, 0)
    if np.issubdtype(np.dtype(dtype), np.integer):
        return np.rint(pts).astype(dtype)
    return pts.astype(dtype)
