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

// Per-warp shared-memory run table of a union: the non-empty cells in
// order, each with its offset in the concatenated candidate list (pre), its
// first sorted position (start) and its coordinates relative to the union
// (7 bits per axis).  pre[nr] is the total.
struct RunTable {
  uint32_t pre[kMaxUnion + 1];
  uint32_t start[kMaxUnion];
  uint32_t cell[kMaxUnion];
};

// Look the union's cells up (one per lane) and fill the run table; returns
// the number of non-empty runs (warp-uniform).  hb is the instance field of
// the hash keys (key_cell in binning.cu).
template <int G>
__device__ __forceinline__ int union_runs(const Union<G>& u,
                                          const unsigned long long* __restrict__ hkeys,
                                          const uint2* __restrict__ hvals, uint32_t hmask,
                                          unsigned long long hb, uint32_t n, int lane,
                                          RunTable& rt) {
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  int nr = 0;
  uint32_t total = 0;
  for (int base = 0; base < u.ncell; base += 32) {
    const int o = base + lane;
    uint32_t st = 0, len = 0, rel = 0;
    if (o < u.ncell) {
      int rem = o;
      uint32_t c[G];
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int q = div_small(rem, u.inv[a]);
        const uint32_t r = (uint32_t)(rem - q * u.w[a]);
        c[a] = (uint32_t)u.lo[a] + r;
        rel |= r << (7 * a);
        rem = q;
      }
      const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, hb | morton<G>(c)), n);
      st = run.x;
      len = run.y - run.x;
    }
    const unsigned m = __ballot_sync(kFull, len > 0);
    uint32_t incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    if (len > 0) {
      const int slot = nr + __popc(m & lanemask_lt);
      rt.pre[slot] = total + incl - len;
      rt.start[slot] = st;
      rt.cell[slot] = rel;
    }
    nr += __popc(m);
    total += __shfl_sync(kFull, incl, 31);
  }
  if (lane == 0) rt.pre[nr] = total;
  __syncwarp();
  return nr;
}

// Run table of a union of at most 64 cells around the queries of one
// segment, ordered by offset class for a multi-pass search over blocks of
// radius 1.  A cell's class is the least number of axes on which it differs
// from the cell of a segment query whose 3^G block contains it (0: a query's
// own cell, 1: a face neighbour, 2: an edge neighbour, ...); cells in no
// query's block get class G + 1 and are left out (no hash lookup either).
// segc holds the segment's nseg distinct query cells.  cend[k] is one past
// the last run of class <= k; returns the number of runs.
template <int G>
__device__ __forceinline__ int union_runs_classed(const Union<G>& u,
                                                  const unsigned long long* __restrict__ hkeys,
                                                  const uint2* __restrict__ hvals, uint32_t hmask,
                                                  unsigned long long hb, uint32_t n, int lane,
                                                  RunTable& rt, const uint32_t (*segc)[G], int nseg,
                                                  int* cend) {
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  uint32_t st[2], len[2], rel[2];
  int cl[2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int o = 32 * b + lane;
    st[b] = len[b] = rel[b] = 0u;
    cl[b] = G + 1;
    if (o < u.ncell) {
      int rem = o;
      uint32_t c[G];
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int q = div_small(rem, u.inv[a]);
        const uint32_t r = (uint32_t)(rem - q * u.w[a]);
        c[a] = (uint32_t)u.lo[a] + r;
        rel[b] |= r << (7 * a);
        rem = q;
      }
      for (int t = 0; t < nseg; ++t) {
        int nnz = 0;
        bool inb = true;
#pragma unroll
        for (int a = 0; a < G; ++a) {
          const int dl = (int)c[a] - (int)segc[t][a];
          inb &= dl >= -1 && dl <= 1;
          nnz += dl != 0;
        }
        if (inb) cl[b] = min(cl[b], nnz);
      }
      if (cl[b] <= G) {
        const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, hb | morton<G>(c)), n);
        st[b] = run.x;
        len[b] = run.y - run.x;
      }
    }
  }
  // slots: by class, then by round and lane; lengths first, offsets below
  int nr = 0;
#pragma unroll
  for (int k = 0; k <= G; ++k) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const bool mine = len[b] > 0 && cl[b] == k;
      const unsigned m = __ballot_sync(kFull, mine);
      if (mine) {
        const int slot = nr + __popc(m & lanemask_lt);
        rt.start[slot] = st[b];
        rt.cell[slot] = rel[b];
        rt.pre[slot] = len[b];
      }
      nr += __popc(m);
    }
    cend[k] = nr;
  }
  __syncwarp();
  uint32_t carry = 0;
  for (int base = 0; base < nr; base += 32) {
    const int sl = base + lane;
    const uint32_t v = sl < nr ? rt.pre[sl] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    if (sl < nr) rt.pre[sl] = carry + incl - v;
    carry += __shfl_sync(kFull, incl, 31);
  }
  if (lane == 0) rt.pre[nr] = carry;
  __syncwarp();
  return nr;
}

// Copy candidates [w0, w1) of the concatenated list into the window: lane l
// copies candidates w0 + l, w0 + l + 32, ...; all loads of a window are
// independent, so the warp keeps many of them in flight.
template <int DP, bool KEYS>
__device__ __forceinline__ void stage_runs(const RunTable& rt, int nr, uint32_t w0, uint32_t w1,
                                           const float* __restrict__ spts,
                                           const unsigned long long* __restrict__ skey,
                                           float* __restrict__ wpts,
                                           unsigned long long* __restrict__ wkey, int lane) {
  // first run holding candidate w0 + lane
  int lo = 0, hi = nr - 1;
  const uint32_t e0 = w0 + lane;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rt.pre[mid] <= e0) lo = mid;
    else hi = mid - 1;
  }
  int r = lo;
  for (uint32_t e = e0; e < w1; e += 32) {
    while (r + 1 < nr && rt.pre[r + 1] <= e) ++r;
    const uint32_t src = rt.start[r] + (e - rt.pre[r]);
    const uint32_t dst = e - w0;
    if constexpr (DP == 2) {
      reinterpret_cast<float2*>(wpts)[dst] = __ldg(reinterpret_cast<const float2*>(spts) + src);
    } else if constexpr (DP == 4) {
      reinterpret_cast<float4*>(wpts)[dst] = __ldg(reinterpret_cast<const float4*>(spts) + src);
    } else {
      const float4* s4 = reinterpret_cast<const float4*>(spts) + 2 * (size_t)src;
      float4* d4 = reinterpret_cast<float4*>(wpts) + 2 * (size_t)dst;
      d4[0] = __ldg(s4);
      d4[1] = __ldg(s4 + 1);
    }
    if constexpr (KEYS) wkey[dst] = __ldg(skey + src);
  }
}

// Visit the runs of window [w0, w1): visit(i0, i1, cell[G]) with window
// indices [i0, i1), warp-uniform.
template <int G, typename Visit>
__device__ __forceinline__ void for_window_runs(const RunTable& rt, int nr, const Union<G>& u,
                                                uint32_t w0, uint32_t w1, Visit visit) {
  for (int r = 0; r < nr; ++r) {
    const uint32_t a = rt.pre[r], b = rt.pre[r + 1];
    if (b <= w0) continue;
    if (a >= w1) break;
    uint32_t c[G];
    const uint32_t rel = rt.cell[r];
#pragma unroll
    for (int x = 0; x < G; ++x) c[x] = (uint32_t)u.lo[x] + ((rel >> (7 * x)) & 127u);
    visit((a > w0 ? a : w0) - w0, (b < w1 ? b : w1) - w0, c);
  }
}

// Copy the runs of `src` for which keep(cell) (warp-uniform) holds into
// `dst`, recomputing the offsets; returns the number kept.
template <int G, typename Keep>
__device__ __forceinline__ int filter_runs(const RunTable& src, int nr, const Union<G>& u,
                                           RunTable& dst, int lane, Keep keep) {
  int m = 0;
  uint32_t total = 0;
  for (int r = 0; r < nr; ++r) {
    uint32_t c[G];
    const uint32_t rel = src.cell[r];
#pragma unroll
    for (int x = 0; x < G; ++x) c[x] = (uint32_t)u.lo[x] + ((rel >> (7 * x)) & 127u);
    if (keep(c)) {
      if (lane == 0) {
        dst.pre[m] = total;
        dst.start[m] = src.start[r];
        dst.cell[m] = rel;
      }
      total += src.pre[r + 1] - src.pre[r];
      ++m;
    }
  }
  if (lane == 0) dst.pre[m] = total;
  __syncwarp();
  return m;
}

template <int DP>
__device__ __forceinline__ Pt<DP> window_pt(const float* __restrict__ wpts, uint32_t i) {
  Pt<DP> p;
  if constexpr (DP == 2) {
    float2 v = reinterpret_cast<const float2*>(wpts)[i];
    p.x[0] = v.x; p.x[1] = v.y;
  } else if constexpr (DP == 4) {
    float4 v = reinterpret_cast<const float4*>(wpts)[i];
    p.x[0] = v.x; p.x[1] = v.y; p.x[2] = v.z; p.x[3] = v.w;
  } else {
    const float4* q = reinterpret_cast<const float4*>(wpts) + 2 * (size_t)i;
    float4 a = q[0], b = q[1];
    p.x[0] = a.x; p.x[1] = a.y; p.x[2] = a.z; p.x[3] = a.w;
    p.x[4] = b.x; p.x[5] = b.y; p.x[6] = b.z; p.x[7] = b.w;
  }
  return p;
}

// Block of radius R around cell c0, clipped to the grid.
template <int G>
__device__ __forceinline__ void block_union(const uint32_t* c0, int R, int cmax, Union<G>& u) {
  int n = 1;
#pragma unroll
  for (int a = 0; a < G; ++a) {
    const int lo = max((int)c0[a] - R, 0);
    const int hi = min((int)c0[a] + R, cmax);
    u.lo[a] = lo;
    u.w[a] = hi - lo + 1;
    u.inv[a] = (65536 + u.w[a] - 1) / u.w[a];
    n *= u.w[a];
  }
  u.ncell = n;
}

// This lane's candidates w0 + lane + 32 v (v < V) of the run table, NaN
// coordinates past the end (a NaN distance fails every comparison); with
// KEYS also their order keys (0 past the end: below every query's key).
template <int DP, int V, bool KEYS = false>
__device__ __forceinline__ void load_window(const RunTable& rt, int nr, uint32_t w0, uint32_t total,
                                            const float* __restrict__ spts, int lane, Pt<DP>* cand,
                                            const unsigned long long* __restrict__ skey = nullptr,
                                            unsigned long long* ck = nullptr) {
  const uint32_t e0 = w0 + lane;
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rt.pre[mid] <= e0) lo = mid;
    else hi = mid - 1;
  }
  int r = lo;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const uint32_t e = e0 + 32u * v;
    if (w0 + 32u * v >= total) break;  // no lane has a candidate in this slot or later
    if (e < total) {
      while (r + 1 < nr && rt.pre[r + 1] <= e) ++r;
      const uint32_t src = rt.start[r] + (e - rt.pre[r]);
      cand[v] = load_pt<DP>(spts, src);
      if constexpr (KEYS) ck[v] = __ldg(skey + src);
    } else {
#pragma unroll
      for (int a = 0; a < DP; ++a) cand[v].x[a] = __int_as_float(0x7fffffff);
      if constexpr (KEYS) ck[v] = 0ull;
    }
  }
}

// load_window with the sorted position of every candidate (0xffffffff past
// the end).
template <int DP, int V>
__device__ __forceinline__ void load_window_pos(const RunTable& rt, int nr, uint32_t w0, uint32_t total,
                                                const float* __restrict__ spts, int lane, Pt<DP>* cand,
                                                uint32_t* pos) {
  const uint32_t e0 = w0 + lane;
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rt.pre[mid] <= e0) lo = mid;
    else hi = mid - 1;
  }
  int r = lo;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const uint32_t e = e0 + 32u * v;
    pos[v] = 0xffffffffu;
    if (w0 + 32u * v >= total) break;
    if (e < total) {
      while (r + 1 < nr && rt.pre[r + 1] <= e) ++r;
      const uint32_t src = rt.start[r] + (e - rt.pre[r]);
      cand[v] = load_pt<DP>(spts, src);
      pos[v] = src;
    } else {
#pragma unroll
      for (int a = 0; a < DP; ++a) cand[v].x[a] = __int_as_float(0x7fffffff);
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

// A segment of the chunk for the segment layouts: from lane s, the longest
// run of whole cells (at least the first cell's lanes) whose bounding box,
// grown by R and clipped to the grid, holds at most max_cells cells; u is set
// to that union (it contains the block of every query of the segment, so a
// search over it sees every point a query's own block holds).  max_cells <= 0
// or a first block larger than max_cells: the first cell alone and its block.
// The union only grows with the segment, so the ends that fit form a prefix.
template <int G>
__device__ __forceinline__ int super_segment(unsigned long long mycell, bool valid, int s, int nvalid,
                                             int R, int cmax, int max_cells, int lane, Union<G>& u) {
  const unsigned long long cell = __shfl_sync(kFull, mycell, s);
  const int e1 = s + __popc(__ballot_sync(kFull, valid && mycell == cell));
  int last = e1 - 1;
  int lo[G], hi[G];
  if (max_cells > 0 && e1 < nvalid) {
    uint32_t mc[G];
    unmorton<G>(valid ? mycell : cell, mc);
    const bool in = valid && lane >= s;
#pragma unroll
    for (int a = 0; a < G; ++a) {
      lo[a] = in ? (int)mc[a] : 0x7fffffff;
      hi[a] = in ? (int)mc[a] : -1;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int tl = __shfl_up_sync(kFull, lo[a], d);
        const int th = __shfl_up_sync(kFull, hi[a], d);
        if (lane >= d) {
          lo[a] = min(lo[a], tl);
          hi[a] = max(hi[a], th);
        }
      }
    }
    long long size = 1;
#pragma unroll
    for (int a = 0; a < G; ++a) size *= (long long)(min(hi[a] + R, cmax) - max(lo[a] - R, 0) + 1);
    const unsigned long long next = __shfl_down_sync(kFull, mycell, 1);
    const bool cell_end = valid && lane >= e1 - 1 && (lane + 1 >= nvalid || next != mycell);
    const unsigned ok = __ballot_sync(kFull, cell_end && size <= (long long)max_cells);
    if (ok & (1u << (e1 - 1))) last = 31 - __clz((int)ok);
  }
  if (last == e1 - 1) {  // the first cell and its block
    uint32_t c0[G];
    unmorton<G>(cell, c0);
    block_union<G>(c0, R, cmax, u);
    return e1;
  }
  int n = 1;
#pragma unroll
  for (int a = 0; a < G; ++a) {
    const int l = max(__shfl_sync(kFull, lo[a], last) - R, 0);
    const int h = min(__shfl_sync(kFull, hi[a], last) + R, cmax);
    u.lo[a] = l;
    u.w[a] = h - l + 1;
    u.inv[a] = (65536 + u.w[a] - 1) / u.w[a];
    n *= u.w[a];
  }
  u.ncell = n;
  return last + 1;
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
