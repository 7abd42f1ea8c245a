// block.cuh -- warp-cooperative visits of the grid blocks of 32 queries.
//
// Work layout shared by the density and near-dependent kernels: a warp owns
// 32 consecutive Morton-sorted points, one query per lane.  Query q needs the
// points of the (2R+1)^g level-k cells around its own cell ("its block").
// The warp takes the bounding box of its queries' cells, grows it by R cells
// (the "union"), looks the union's cells up in the occupied-cell hash in
// parallel (one cell per lane), and then streams every non-empty cell's run of
// sorted points with all lanes reading the same point (one broadcast load).
// A lane whose block does not contain the cell masks it out, so every query
// sees exactly the points of its own block.  When the union would exceed
// kMaxUnion cells (the 32 points straddle a jump of the Morton curve), the
// warp splits its points into runs of equal cell and visits each separately.
#pragma once

#include "dpc_device.cuh"

namespace dpc {

constexpr int kMaxUnion = 128;
constexpr unsigned kFull = 0xffffffffu;

// floor(x / w) for 0 <= x < 128, 1 <= w <= 128: x * ceil(2^16 / w) >> 16 is exact
// there (the rounding term x * (w * ceil(2^16 / w) - 2^16) stays below 2^16 / 4).
__device__ __forceinline__ int div_small(int x, int inv) { return (x * inv) >> 16; }

template <int G>
struct Union {
  int lo[G];   // first cell of the union per axis
  int w[G];    // extent per axis
  int inv[G];  // ceil(2^16 / w)
  int ncell;
};

// Bounding box of the cells of the active lanes, grown by R and clipped to
// the grid.  Returns false (union unusable) if it holds more than kMaxUnion
// cells.
template <int G>
__device__ __forceinline__ bool make_union(const uint32_t* c0, bool active, int R, int cmax,
                                           Union<G>& u) {
  int n = 1;
  if (!__any_sync(kFull, active)) {  // no query: an empty union
    u.ncell = 0;
    return true;
  }
#pragma unroll
  for (int a = 0; a < G; ++a) {
    int mn = active ? (int)c0[a] : 0x7fffffff;
    int mx = active ? (int)c0[a] : -1;
    mn = __reduce_min_sync(kFull, mn);
    mx = __reduce_max_sync(kFull, mx);
    const int lo = max(mn - R, 0);
    const int hi = min(mx + R, cmax);
    u.lo[a] = lo;
    u.w[a] = hi - lo + 1;
    u.inv[a] = (65536 + u.w[a] - 1) / u.w[a];
    n *= u.w[a];
    if (n > kMaxUnion) {
      n = kMaxUnion + 1;
    }
  }
  u.ncell = n;
  return n <= kMaxUnion;
}

// Visit every non-empty cell of the union: visit(start, len, cell[G]) is
// called by all lanes with the same arguments (warp-uniform).
template <int G, typename Visit>
__device__ __forceinline__ void for_union_cells(const Union<G>& u,
                                                const unsigned long long* __restrict__ hkeys,
                                                const uint2* __restrict__ hvals, uint32_t hmask,
                                                uint32_t n, int lane, Visit visit) {
  for (int base = 0; base < u.ncell; base += 32) {
    const int o = base + lane;
    uint32_t st = 0, len = 0;
    uint32_t c[G];
#pragma unroll
    for (int a = 0; a < G; ++a) c[a] = 0;
    if (o < u.ncell) {
      int rem = o;
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int q = div_small(rem, u.inv[a]);
        c[a] = (uint32_t)(u.lo[a] + rem - q * u.w[a]);
        rem = q;
      }
      const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, morton<G>(c)), n);
      st = run.x;
      len = run.y - run.x;
    }
    unsigned mask = __ballot_sync(kFull, len > 0);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      uint32_t cj[G];
#pragma unroll
      for (int a = 0; a < G; ++a) cj[a] = __shfl_sync(kFull, c[a], j);
      visit(__shfl_sync(kFull, st, j), __shfl_sync(kFull, len, j), cj);
    }
  }
}

// Does the block of radius R around cell c0 contain cell c?
template <int G>
__device__ __forceinline__ bool in_block(const uint32_t* c0, const uint32_t* c, int R) {
  bool in = true;
#pragma unroll
  for (int a = 0; a < G; ++a) in &= abs((int)c[a] - (int)c0[a]) <= R;
  return in;
}

// The warp's groups of lanes: the whole chunk if its union is small enough,
// else one group per cell.  group(active, union) is called for each group.
// `valid` marks lanes holding a point (a prefix of the warp), `active` the
// queries to answer (a subset of them).
template <int G, typename Group>
__device__ __forceinline__ void for_groups(const unsigned long long mycell, const uint32_t* c0,
                                           bool valid, bool active, int nvalid, int R, int cmax,
                                           int lane, Group group) {
  Union<G> u;
  if (make_union<G>(c0, active, R, cmax, u)) {
    group(active, u);
    return;
  }
  int s = 0;
  while (s < nvalid) {
    const unsigned long long cell = __shfl_sync(kFull, mycell, s);
    const bool same = valid && mycell == cell;  // lanes s .. e-1 (sorted order)
    const int e = s + __popc(__ballot_sync(kFull, same));
    const bool act = same && active;
    if (__any_sync(kFull, act)) {
      make_union<G>(c0, act, R, cmax, u);  // one cell: (2R+1)^g <= kMaxUnion
      group(act, u);
    }
    s = e;
  }
}

}  // namespace dpc
