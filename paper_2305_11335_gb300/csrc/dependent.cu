// dependent.cu -- lambda_i (the nearest point of higher order) and
// delta_i = D(x_i, lambda_i) (Definitions 2-3).
//
// The paper runs one priority nearest-neighbour query per point in parallel
// (Algorithm 1) on a priority search kd-tree.  Here each query runs in two
// phases:
//   near  the grid block around the point's cell (the cells the density
//         used), streamed by the warp with one query per lane (block.cuh).
//         If the best candidate is closer than anything outside the block
//         can be, and no other candidate is within the float32 error band
//         of it, the query is settled; this holds for most points, since a
//         point's dependent point is usually within d_cut.
//   far   the remaining queries (local density maxima, isolated points, near
//         ties) walk the radix tree (tree.cu) depth first, nearer child
//         first, skipping subtrees whose largest key is not above the query's
//         key or whose box is farther than the best candidate so far (the
//         pruning of Section 4.1.2).
//
// Exactness.  Candidates are compared on their float32 distance s32; the
// winner of the binary64 order (s64, id) -- the write-min of Section 3.2 --
// is certainly the float32 winner unless another candidate lies within the
// float32 error band of it.  The query tracks the smallest and second
// smallest s32; when the second is inside the band the candidates inside it
// are re-ranked in binary64 (rare: exact ties and near ties).  delta is
// always sqrt of the winner's binary64 distance.  In FP64 mode every
// candidate is compared in binary64 directly.
#include <cmath>
#include <type_traits>

#include "block.cuh"
#include "internal.h"

namespace dpc {

namespace {

constexpr int kFarThreads = 128;
constexpr int kStack = 128;
constexpr int kWarpStack = 1024;  // shared stack entries per warp (far phase, round 2)
constexpr uint32_t kFarBudget = 128;  // node expansions per query in round 1
constexpr int kNearWarps = 4;
constexpr int kNearThreads = kNearWarps * 32;

__device__ __forceinline__ float band_of(float s, float mul, float add) {
  return __fadd_ru(__fmul_ru(s, mul), add);
}

// A region whose float lower bound lbs (already 1e-5 below the true squared
// distance) exceeds `bound` by this much holds no candidate with s32 <= bound:
// the margin dominates the absolute float32 error term of tiny distances.
constexpr float kPruneAbs = 1e-33f;
__device__ __forceinline__ bool beyond(float lbs, float bound) {
  return lbs > __fadd_ru(bound, kPruneAbs);
}

// Running minimum of (s, id), the second smallest s, and the sorted position
// of the minimum (tree phase).
template <typename S>
struct Best {
  S s1, s2;
  uint32_t o1;   // id of the best
  uint32_t t1;   // sorted position of the best
  __device__ __forceinline__ void init() {
    s1 = (S)INFINITY;
    s2 = (S)INFINITY;
    o1 = 0xffffffffu;
    t1 = 0xffffffffu;
  }
  __device__ __forceinline__ void add(S s, uint32_t o, uint32_t t) {
    if (s < s1 || (s == s1 && o < o1)) {
      s2 = s1;
      s1 = s;
      o1 = o;
      t1 = t;
    } else if (s < s2) {
      s2 = s;
    }
  }
  // union over the warp's lanes (every lane ends with the same summary)
  __device__ __forceinline__ void merge_warp() {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const S b1 = __shfl_xor_sync(kFull, s1, m);
      const uint32_t bo = __shfl_xor_sync(kFull, o1, m);
      const S b2 = __shfl_xor_sync(kFull, s2, m);
      const uint32_t bt = __shfl_xor_sync(kFull, t1, m);
      if (b1 < s1 || (b1 == s1 && bo < o1)) {
        s2 = s1 < b2 ? s1 : b2;
        s1 = b1;
        o1 = bo;
        t1 = bt;
      } else {
        s2 = s2 < b1 ? s2 : b1;
      }
    }
  }
};

// Exact binary64 argmin over (s64, id).
struct Exact {
  double s;
  uint32_t o;
  __device__ __forceinline__ void init() {
    s = INFINITY;
    o = 0xffffffffu;
  }
  __device__ __forceinline__ void add(double v, uint32_t id) {
    if (v < s || (v == s && id < o)) {
      s = v;
      o = id;
    }
  }
  __device__ __forceinline__ void merge_warp() {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) add(__shfl_xor_sync(kFull, s, m), __shfl_xor_sync(kFull, o, m));
  }
};

// Conservative squared lower bound, in fine units, between the query and a box
// of fine indices [lo, hi] on each axis (a point of fine index c lies in
// [c - 0.5, c + 1.5) fine units; the query's float position is within 1/8).
__device__ __forceinline__ float lb_axis(float lo, float hi, float u) {
  return fmaxf(fmaxf(lo - 1.f - u, u - hi - 2.f), 0.f);
}

// ---------------------------------------------------------------------------
// near phase

// Smallest and second smallest float32 distance of a candidate set, and the id
// of a candidate at the smallest.  Two candidates at the same smallest
// distance leave s2 == s1, which the caller treats as ambiguous and resolves
// in binary64 later, so ties need no id order here.
struct Min2 {
  float s1, s2;
  uint32_t o1;
  __device__ __forceinline__ void init() {
    s1 = s2 = INFINITY;
    o1 = 0xffffffffu;
  }
  __device__ __forceinline__ void add(float v, uint32_t id) {
    s2 = fminf(s2, fmaxf(s1, v));
    o1 = v < s1 ? id : o1;
    s1 = fminf(s1, v);
  }
};

// Coordinates of point `id` of the instance whose coordinates start at
// element `coord` of the caller's input (the same float values the sorted copy
// holds: int32 inputs are exact in float32 by the range check).
template <int DP>
__device__ __forceinline__ Pt<DP> input_pt(const void* __restrict__ pts, int dtype, uint64_t coord,
                                           int d, uint32_t id) {
  Pt<DP> p;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
    float v = 0.f;
    if (a < d) {
      const size_t e = coord + (size_t)id * d + a;
      v = dtype == 0 ? (float)__ldg((const int32_t*)pts + e) : __ldg((const float*)pts + e);
    }
    p.x[a] = v;
  }
  return p;
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kNearThreads)
k_dep_near(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
           const unsigned long long* __restrict__ skey, ClassView cv, int32_t rho_skip,
           const void* __restrict__ pts, int dtype, const CutGeom* __restrict__ cuts,
           const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
           const uint2* __restrict__ hvals, int32_t* __restrict__ lambda,
           double* __restrict__ delta, FarQueue q, Counters* ctr) {
  constexpr int kNearCap = DP == 8 ? 128 : 256;
  __shared__ __align__(16) float s_pts[kNearWarps * kNearCap * DP];
  __shared__ unsigned long long s_key[kNearWarps * kNearCap];
  __shared__ RunTable s_rt[kNearWarps];
  __shared__ RunTable s_rt2[kNearWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* wpts = s_pts + wib * kNearCap * DP;
  unsigned long long* wkey = s_key + wib * kNearCap;
  RunTable& rt = s_rt[wib];
  RunTable& rt2 = s_rt2[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (uint32_t ch = blockIdx.x * kNearWarps + wib; ch < cv.nchunk; ch += gridDim.x * kNearWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const InstDev I = cv.instance(inst);
    const GridGeom* geom = cv.geom + inst;
    const CutGeom& C = cuts[inst];
    const float f2lo = geom->f2 * (1.f - 1e-5f);
    const double inv_f = geom->inv_f;
    double org[G];
#pragma unroll
    for (int a = 0; a < G; ++a) org[a] = geom->org[a];
    const int k = C.k;
    const float cell_fine = (float)(1u << k);
    const int R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (geom->B - k)) - 1;
    const float bmul = C.band_mul, badd = C.band_add;
    const float far32 = C.far32;
    const double far64 = C.far64;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    Pt<DP> me;
#pragma unroll
    for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
    unsigned long long K = ~0ull;
    if (valid) {
      me = load_pt<DP>(spts, p);
      K = skey[p];
    }
    const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
    uint32_t c0[G];
    unmorton<G>(valid ? mycell : 0ull, c0);
    const bool skip = valid && (int32_t)(K >> 32) < max(rho_skip, C.skip);
    const int nvalid = (int)min(32u, end - p0);
    Min2 acc;
    acc.init();
    Exact acc64;
    acc64.init();
    // the query's position in fine units, for cell lower bounds
    float uq[G];
#pragma unroll
    for (int a = 0; a < G; ++a) uq[a] = valid ? (float)(((double)me.x[a] - org[a]) * inv_f) : 0.f;
    for_groups<G>(mycell, c0, valid, valid && !skip, nvalid, R, cmax, lane,
                  [&](bool act, const Union<G>& u) {
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      // scan every run of a table, staged window by window
      auto scan = [&](const RunTable& tab, int nt) {
        const uint32_t total = tab.pre[nt];
        for (uint32_t w0 = 0; w0 < total; w0 += kNearCap) {
          const uint32_t w1 = min(total, w0 + (uint32_t)kNearCap);
          __syncwarp();
          stage_runs<DP, true>(tab, nt, w0, w1, spts, skey, wpts, wkey, lane);
          __syncwarp();
          for_window_runs<G>(tab, nt, u, w0, w1, [&](uint32_t i0, uint32_t i1, const uint32_t* cc) {
            const bool need = act && in_block<G>(c0, cc, R);
            if (!__any_sync(kFull, need)) return;
            // a lane outside this cell's block takes no candidate: no key exceeds ~0
            const unsigned long long Kl = need ? K : ~0ull;
#pragma unroll 4
            for (uint32_t i = i0; i < i1; ++i) {
              const unsigned long long kt = wkey[i];
              const Pt<DP> x = window_pt<DP>(wpts, i);
              if constexpr (F64) {
                if (kt > Kl) acc64.add(dist64<DP>(me, x), key_id(kt));
              } else {
                const float d32 = dist32<DP>(me, x);
                acc.add(kt > Kl ? d32 : INFINITY, key_id(kt));
              }
            }
          });
        }
        __syncwarp();
      };
      auto own = [&](const uint32_t* cc) {
        bool same = act;
#pragma unroll
        for (int a = 0; a < G; ++a) same &= cc[a] == c0[a];
        return __any_sync(kFull, same) != 0;
      };
      // a small union: one pass over everything
      if (rt.pre[nr] <= 4u * kNearCap) {
        scan(rt, nr);
        return;
      }
      // pass 1: the cells holding the group's own queries -- unless they hold
      // too few points to bound the search, then one pass over everything
      const int n1 = filter_runs<G>(rt, nr, u, rt2, lane, own);
      if (rt2.pre[n1] < 96u) {
        scan(rt, nr);
        return;
      }
      scan(rt2, n1);
      // pass 2: the other cells of the blocks that can still hold a point
      // closer than some lane's best (a conservative lower bound decides)
      scan(rt2, filter_runs<G>(rt, nr, u, rt2, lane, [&](const uint32_t* cc) {
        if (own(cc)) return false;
        bool need = act && in_block<G>(c0, cc, R);
        if (need) {
          float lb2 = 0.f;
#pragma unroll
          for (int a = 0; a < G; ++a) {
            const float lo = (float)cc[a] * cell_fine;
            const float l = lb_axis(lo, lo + cell_fine - 1.f, uq[a]);
            lb2 = fmaf(l, l, lb2);
          }
          const float lbs = lb2 * f2lo;
          if constexpr (F64) need = (double)lbs <= acc64.s;
          else need = !beyond(lbs, band_of(acc.s1, bmul, badd));
        }
        return __any_sync(kFull, need) != 0;
      }));
    });

    bool settled = false;
    float s1 = INFINITY;
    if (valid && !skip) {
      const uint32_t id = key_id(K);
      if constexpr (F64) {
        settled = acc64.o != 0xffffffffu && acc64.s < far64;
        if (settled) {
          lambda[id] = (int32_t)(acc64.o - (uint32_t)I.out);
          delta[id] = sqrt(acc64.s);
        }
      } else if (acc.o1 != 0xffffffffu) {
        s1 = acc.s1;
        const float bnd = band_of(s1, bmul, badd);
        settled = bnd < far32 && acc.s2 > bnd;
        if (settled) {
          const uint32_t o = acc.o1 - (uint32_t)I.out;
          lambda[id] = (int32_t)o;
          delta[id] = sqrt(dist64<DP>(me, input_pt<DP>(pts, dtype, I.coord, I.d, o)));
        }
      }
    } else if (valid) {
      const uint32_t id = key_id(K);
      lambda[id] = -1;
      delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: skipped
    }
    // unsettled queries (nothing near, or a near tie) go to the far phase
    const bool push = valid && !skip && !settled;
    const unsigned pm = __ballot_sync(kFull, push);
    uint32_t base = 0;
    if (lane == 0 && pm) base = atomicAdd(&ctr->queue_n, (unsigned)__popc(pm));
    base = __shfl_sync(kFull, base, 0);
    if (push) {
      const uint32_t slot = base + __popc(pm & lanemask_lt);
      q.pos[slot] = p;
      if constexpr (F64) q.s1d[slot] = acc64.s;
      else q.s1[slot] = s1;
    }
  }
}

// Segment form of the near phase (the work layout of k_density_seg): the
// chunk's points are split into segments of equal cell; for each segment the
// block's candidates (and their order keys) are spread over the lanes, and for
// every query of the segment each lane keeps the two smallest float32
// distances among its higher candidates, merged over the warp with three
// reductions.  Lane j collects the running best of the chunk's query j, then
// settles it or queues it for the far phase exactly as k_dep_near does.
// With radius-1 blocks in 2 or 3 gridded dimensions (float32) the block's
// cells are taken in order of the number of axes on which they differ from a
// query's own cell, and between windows a query whose winner is already
// certified against every cell left leaves the sweep (on c3 73% of the
// queries are certified before the cells that differ on all three axes).
// 4 candidate slots per lane at 5 blocks per SM: the kernel is latency-bound,
// and resident warps pay more than longer windows.

template <int DP>
constexpr int near_seg_v() { return DP == 8 ? 4 : (DP == 4 ? 4 : 8); }

// Merges the candidate summary (a1 smallest, a2 second smallest, ao an id at
// a1) into a running one; equal smallest distances leave s2 == s1.
__device__ __forceinline__ void min2_merge(Min2& m, float a1, float a2, uint32_t ao) {
  const float hi1 = fmaxf(m.s1, a1);
  m.s2 = fminf(fminf(m.s2, a2), hi1);
  m.o1 = a1 < m.s1 ? ao : m.o1;
  m.s1 = fminf(m.s1, a1);
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kNearThreads, 5)
k_dep_near_seg(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
               const unsigned long long* __restrict__ skey, ClassView cv, int32_t rho_skip,
               const void* __restrict__ pts, int dtype, const CutGeom* __restrict__ cuts,
               const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
               const uint2* __restrict__ hvals, int32_t* __restrict__ lambda,
               double* __restrict__ delta, FarQueue q, Counters* ctr, int seg_cells) {
  constexpr int ND = real_dims<DP, G>();  // coordinates that can be nonzero
  constexpr int V = near_seg_v<DP>();
  constexpr uint32_t W = 32u * V;
  __shared__ RunTable s_rt[kNearWarps];
  __shared__ RunTable s_rt2[kNearWarps];
  __shared__ uint32_t s_segc[kNearWarps][32][G];  // distinct query cells of a segment
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  RunTable& rt = s_rt[wib];
  RunTable& rt2 = s_rt2[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (uint32_t ch = blockIdx.x * kNearWarps + wib; ch < cv.nchunk; ch += gridDim.x * kNearWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const InstDev I = cv.instance(inst);
    const CutGeom& C = cuts[inst];
    const int k = C.k;
    const int R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const float bmul = C.band_mul, badd = C.band_add;
    const float far32 = C.far32;
    const double far64 = C.far64;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    unsigned long long K = ~0ull;
    if (valid) K = skey[p];
    const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
    const bool skip = valid && (int32_t)(K >> 32) < max(rho_skip, C.skip);
    const int nvalid = (int)min(32u, end - p0);
    // this lane's query in fine units, for the cell lower bounds of pass 2
    const GridGeom* geom = cv.geom + inst;
    const float f2lo = geom->f2 * (1.f - 1e-5f);
    const float cell_fine = (float)(1u << k);
    float uq[G];
    {
      const Pt<DP> me = valid ? load_pt<DP>(spts, p) : Pt<DP>{};
#pragma unroll
      for (int a = 0; a < G; ++a)
        uq[a] = valid ? (float)(((double)me.x[a] - geom->org[a]) * geom->inv_f) : 0.f;
    }
    // multi-pass search (float32, radius-1 blocks of 2 or 3 gridded axes):
    // this lane's cell, and squared lower bounds of the distance from its
    // query to any cell differing from its own on at least 2 (lbc[0]) or 3
    // (lbc[1]) axes: the sums of the smallest squared gaps to the cell's faces
    constexpr bool kClassed = !F64 && (G == 2 || G == 3);
    float lbc[2] = {0.f, 0.f};
    if constexpr (kClassed) {
      uint32_t cown[G];
      unmorton<G>(valid ? mycell : 0ull, cown);
      float g2[G];
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const float lo = (float)cown[a] * cell_fine;
        const float gp = fmaxf(fminf(uq[a] - lo - 1.f, lo + cell_fine - 1.f - uq[a]), 0.f);
        g2[a] = gp * gp;
      }
      if constexpr (G == 2) {
        lbc[0] = (g2[0] + g2[1]) * f2lo;
      } else {
        const float mx = fmaxf(fmaxf(g2[0], g2[1]), g2[2]);
        const float sum = g2[0] + g2[1] + g2[2];
        lbc[0] = (sum - mx) * f2lo;
        lbc[1] = sum * f2lo;
      }
    }
    Min2 best;  // lane j: query p0 + j
    best.init();
    Exact best64;
    best64.init();
    int s = 0;
    while (s < nvalid) {
      const unsigned long long cell = __shfl_sync(kFull, mycell, s);
      Union<G> u;
      const int e = super_segment<G>(mycell, valid, s, nvalid, R, cmax, seg_cells, lane, u);
      const unsigned seg = (e >= 32 ? 0xffffffffu : ((1u << e) - 1u)) & ~((1u << s) - 1u);  // lanes s .. e-1
      // one cell only: the own-cell-first passes below apply
      const bool single = (__ballot_sync(kFull, valid && mycell == cell) & seg) == seg;
      if (__ballot_sync(kFull, valid && !skip) & seg) {
        uint32_t c0[G];
        unmorton<G>(cell, c0);
        // the segment's queries to answer
        const unsigned qall = seg & __ballot_sync(kFull, valid && !skip);
        // class-ordered run table (see below): runs [0, ce1) hold the cells
        // differing from some query's own cell on at most one axis, [ce1,
        // ce2) those differing on two
        bool classed = false;
        int ce1 = 0, ce2 = 0;
        // candidates [P0, total) of a run table, window by window, for the
        // queries of mask qm
        auto scan = [&](const RunTable& tab, int ntab, uint32_t P0, uint32_t total, unsigned qm) {
        for (uint32_t w0 = P0; w0 < total; w0 += W) {
          Pt<DP> cand[V];
          unsigned long long ck[V];
          load_window<DP, V, true>(tab, ntab, w0, total, spts, lane, cand, skey, ck);
          const int vn = (int)min((uint32_t)V, (total - w0 + 31u) / 32u);
          // two queries per pass over the lane's candidates (independent chains)
          for (unsigned m = qm; m;) {
            const int j = __ffs(m) - 1;
            m &= m - 1u;
            const bool two = m != 0u;
            const int jb = two ? __ffs(m) - 1 : j;
            if (two) m &= m - 1u;
            const unsigned long long Ka = __shfl_sync(kFull, K, j);
            const unsigned long long Kb = __shfl_sync(kFull, K, jb);
            constexpr bool act_a = true;
            const bool act_b = two;
            const Pt<DP> xa = load_pt<DP>(spts, p0 + j);
            const Pt<DP> xb = load_pt<DP>(spts, p0 + jb);
            if constexpr (F64) {
              Exact ea, eb;
              ea.init();
              eb.init();
#pragma unroll
              for (int v = 0; v < V; ++v) {
                if (v >= vn) break;
                if (ck[v] > Ka) ea.add(dist64<DP, ND>(xa, cand[v]), key_id(ck[v]));
                if (ck[v] > Kb) eb.add(dist64<DP, ND>(xb, cand[v]), key_id(ck[v]));
              }
              ea.merge_warp();
              eb.merge_warp();
              if (act_a && lane == j) best64.add(ea.s, ea.o);
              if (act_b && lane == jb) best64.add(eb.s, eb.o);
            } else {
              Min2 ma, mb;
              ma.init();
              mb.init();
#pragma unroll
              for (int v = 0; v < V; ++v) {
                if (v >= vn) break;
                const float da = dist32<DP, ND>(xa, cand[v]);
                const float db = dist32<DP, ND>(xb, cand[v]);
                const uint32_t id = key_id(ck[v]);
                ma.add(ck[v] > Ka ? da : INFINITY, id);
                mb.add(ck[v] > Kb ? db : INFINITY, id);
              }
              // per query: the warp's two smallest and an id at the smallest
              auto warp_min2 = [&](const Min2& m, float& g1, float& g2, uint32_t& go) {
                g1 = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(m.s1)));
                const unsigned at = __ballot_sync(kFull, m.s1 == g1);
                go = __reduce_min_sync(kFull, m.s1 == g1 ? m.o1 : 0xffffffffu);
                g2 = __popc(at) > 1
                         ? g1
                         : __uint_as_float(
                               __reduce_min_sync(kFull, __float_as_uint(m.s1 == g1 ? m.s2 : m.s1)));
                if (!(g1 < INFINITY)) go = 0xffffffffu;
              };
              float a1, a2, b1, b2;
              uint32_t ao, bo;
              warp_min2(ma, a1, a2, ao);
              warp_min2(mb, b1, b2, bo);
              if (act_a && lane == j) min2_merge(best, a1, a2, ao);
              if (act_b && lane == jb) min2_merge(best, b1, b2, bo);
            }
          }
          if constexpr (kClassed) {
            // class-ordered table: the candidates left all lie in cells that
            // differ from each query's own cell on at least two (three) axes;
            // a query whose winner is certified and closer than every such
            // cell takes no part in the windows left
            const uint32_t nxt = w0 + W;
            if (classed && nxt < total && nxt >= tab.pre[ce1]) {
              const float lb = nxt >= tab.pre[ce2] ? lbc[1] : lbc[0];
              bool done = false;
              if ((qm >> lane) & 1u) {
                if (best.o1 != 0xffffffffu) {
                  const float bnd = band_of(best.s1, bmul, badd);
                  done = bnd < far32 && best.s2 > bnd && beyond(lb, bnd);
                }
              }
              qm &= ~__ballot_sync(kFull, done);
              if (!qm) break;
            }
          }
        }
        };
        if constexpr (kClassed) classed = R == 1 && u.ncell <= 64;
        // Classed (float32, radius-1 blocks of 2 or 3 gridded axes): the
        // union's cells ordered by the least number of axes on which they
        // differ from some query's own cell, one sweep of windows over them,
        // and queries certified early leave it (above).  Cells in no query's
        // block are left out: they lie beyond the far bound of every query.
        // Otherwise dense blocks (more than 8 windows) of one cell: pass 1
        // scans the segment's own cell, pass 2 only the other cells that can
        // still hold a point closer than some query's best (a conservative
        // lower bound decides); any other block: one pass over everything.
        int nr, np;
        if (classed) {
          // the first lane of each cell of the segment (all lanes shuffle)
          const unsigned long long prev = __shfl_up_sync(kFull, mycell, 1);
          const bool head = ((seg >> lane) & 1u) && valid && (lane == s || prev != mycell);
          const unsigned heads = __ballot_sync(kFull, head);
          if (head) {
            uint32_t cc[G];
            unmorton<G>(mycell, cc);
            const int r = __popc(heads & lanemask_lt);
#pragma unroll
            for (int a = 0; a < G; ++a) s_segc[wib][r][a] = cc[a];
          }
          __syncwarp();
          int cend[G + 1];
          nr = union_runs_classed<G>(u, hkeys, hvals, hmask, hb, n, lane, rt, s_segc[wib],
                                     __popc(heads), cend);
          ce1 = cend[1];
          ce2 = cend[2];
          np = 1;
        } else {
          nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
          np = (!single || rt.pre[nr] <= 8u * W) ? 1 : 2;
        }
        auto own = [&](const uint32_t* cc) {
          bool same = true;
#pragma unroll
          for (int a = 0; a < G; ++a) same &= cc[a] == c0[a];
          return same;
        };
        const bool mine = ((seg >> lane) & 1u) && !skip;
        for (int pass = 0; pass < np; ++pass) {
          int ntab = nr;
          const RunTable* tab = &rt;
          if (np == 2) {
            tab = &rt2;
            if (pass == 0) {
              ntab = filter_runs<G>(rt, nr, u, rt2, lane, own);
            } else {
              ntab = filter_runs<G>(rt, nr, u, rt2, lane, [&](const uint32_t* cc) {
                if (own(cc)) return false;
                bool need = mine;
                if (need) {
                  float lb2 = 0.f;
#pragma unroll
                  for (int a = 0; a < G; ++a) {
                    const float lo = (float)cc[a] * cell_fine;
                    const float l = lb_axis(lo, lo + cell_fine - 1.f, uq[a]);
                    lb2 = fmaf(l, l, lb2);
                  }
                  const float lbs = lb2 * f2lo;
                  if constexpr (F64) need = (double)lbs <= best64.s;
                  else need = !beyond(lbs, band_of(best.s1, bmul, badd));
                }
                return __any_sync(kFull, need) != 0;
              });
            }
          }
          scan(*tab, ntab, 0u, tab->pre[ntab], qall);
        }
      }
      s = e;
    }

    bool settled = false;
    float s1 = INFINITY;
    if (valid && !skip) {
      const uint32_t id = key_id(K);
      if constexpr (F64) {
        settled = best64.o != 0xffffffffu && best64.s < far64;
        if (settled) {
          lambda[id] = (int32_t)(best64.o - (uint32_t)I.out);
          delta[id] = sqrt(best64.s);
        }
      } else if (best.o1 != 0xffffffffu) {
        s1 = best.s1;
        const float bnd = band_of(s1, bmul, badd);
        settled = bnd < far32 && best.s2 > bnd;
        if (settled) {
          const uint32_t o = best.o1 - (uint32_t)I.out;
          const Pt<DP> me = load_pt<DP>(spts, p);
          lambda[id] = (int32_t)o;
          delta[id] = sqrt(dist64<DP>(me, input_pt<DP>(pts, dtype, I.coord, I.d, o)));
        }
      }
    } else if (valid) {
      const uint32_t id = key_id(K);
      lambda[id] = -1;
      delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: skipped
    }
    // unsettled queries (nothing near, or a near tie) go to the far phase
    const bool push = valid && !skip && !settled;
    const unsigned pm = __ballot_sync(kFull, push);
    uint32_t base = 0;
    if (lane == 0 && pm) base = atomicAdd(&ctr->queue_n, (unsigned)__popc(pm));
    base = __shfl_sync(kFull, base, 0);
    if (push) {
      const uint32_t slot = base + __popc(pm & lanemask_lt);
      q.pos[slot] = p;
      if constexpr (F64) q.s1d[slot] = best64.s;
      else q.s1[slot] = s1;
    }
  }
}

// Tree layout of the near phase: no block scan; every query (but the skipped
// ones) goes to the tree search with no bound.  Pays off where blocks are
// dense enough that a best-first search of the tree, pruned by maximum key and
// by box distance, visits far fewer points than the block holds.
// One warp per 32-point chunk (the chunk gives the instance, hence its skip
// threshold).
__global__ void k_near_to_far(const unsigned long long* __restrict__ skey, ClassView cv,
                              const CutGeom* __restrict__ cuts, int32_t rho_skip,
                              int32_t* __restrict__ lambda, double* __restrict__ delta, FarQueue q,
                              Counters* ctr) {
  const int lane = threadIdx.x & 31;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  const uint64_t total = (uint64_t)cv.nchunk * 32u;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t inst, p0, end;
    cv.chunk((uint32_t)(e >> 5), inst, p0, end);
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    const unsigned long long K = valid ? skey[p] : 0ull;
    const bool skip = valid && (int32_t)(K >> 32) < max(rho_skip, cuts[inst].skip);
    if (skip) {
      const uint32_t id = key_id(K);
      lambda[id] = -1;
      delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: skipped
    }
    const bool push = valid && !skip;
    const unsigned pm = __ballot_sync(kFull, push);
    uint32_t base = 0;
    if (lane == 0 && pm) base = atomicAdd(&ctr->queue_n, (unsigned)__popc(pm));
    base = __shfl_sync(kFull, base, 0);
    if (push) {
      const uint32_t slot = base + __popc(pm & lanemask_lt);
      q.pos[slot] = p;
      q.s1[slot] = INFINITY;
      q.s1d[slot] = INFINITY;
    }
  }
}

// ---------------------------------------------------------------------------
// far phase: depth-first priority search of the radix tree

// Squared lower bound between the query and the bounding box of a subtree
// (all coordinates; box layout [lo(DP) | hi(DP)] per node, tree.cu), scaled
// 1e-5 down so that it stays below the float32 distance of every point inside
// despite the rounding of this evaluation and of dist32.
template <int DP>
__device__ __forceinline__ float rec_lb2(const ChildRec<DP>& r, int s, const Pt<DP>& x) {
  float lb2 = 0.f;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
    const float l = fmaxf(fmaxf(r.lo[s][a] - x.x[a], x.x[a] - r.hi[s][a]), 0.f);
    lb2 = fmaf(l, l, lb2);
  }
  return lb2 * (1.f - 1e-5f);
}

// A leaf child's point, from its record (its box is the point itself).
template <int DP>
__device__ __forceinline__ Pt<DP> rec_point(const ChildRec<DP>& r, int s) {
  Pt<DP> p;
#pragma unroll
  for (int a = 0; a < DP; ++a) p.x[a] = r.lo[s][a];
  return p;
}

enum { kWalkDone = 0, kWalkBudget = 1, kWalkBad = -1 };

// One thread's depth-first search below internal node `start`, nearer child
// first: every leaf with key > K not excluded by `prune` is passed to
// visit(t, kt, point).  Expanding a node reads its child record alone (the
// children's indices, keys and boxes).  Stops with kWalkBudget after `budget` node expansions, and
// with kWalkBad on a malformed tree or stack overflow (neither happens for a
// tree built by tree.cu: its depth is at most 64 + 32).
template <int DP, typename Prune, typename Visit>
__device__ __noinline__ int tree_walk_from(const Node* __restrict__ nodes,
                                           const float* __restrict__ nbox, uint32_t n,
                                           const unsigned long long* __restrict__ skey,
                                           unsigned long long K, const Pt<DP>& xq,
                                           uint32_t start, uint32_t budget, uint32_t& expanded,
                                           Prune prune, Visit visit) {
  uint32_t stk[kStack];
  float stl[kStack];
  int sp = 0;
  stk[sp] = start;
  stl[sp] = 0.f;
  ++sp;
  while (sp > 0) {
    --sp;
    const uint32_t ni = stk[sp];
    if (prune(stl[sp])) continue;
    if (ni + 1 >= n) return kWalkBad;
    if (expanded >= budget) return kWalkBudget;
    ++expanded;
    const ChildRec<DP> r = load_rec<DP>(nbox, ni);
    uint32_t keep[2];
    float keepl[2];
    int nk = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t c = r.child[s];
      if (r.key[s] <= K) continue;  // nothing of higher key below
      if (c & kLeafBit) {
        if ((c & ~kLeafBit) >= n) return kWalkBad;
        visit(c & ~kLeafBit, r.key[s], rec_point<DP>(r, s));
      } else {
        const float lbs = rec_lb2<DP>(r, s, xq);
        if (prune(lbs)) continue;
        keep[nk] = c;
        keepl[nk] = lbs;
        ++nk;
      }
    }
    if (sp + nk > kStack) return kWalkBad;
    if (nk == 2 && keepl[0] < keepl[1]) {  // push the farther child first
      stk[sp] = keep[1]; stl[sp] = keepl[1]; ++sp;
      stk[sp] = keep[0]; stl[sp] = keepl[0]; ++sp;
    } else {
      for (int s = 0; s < nk; ++s) { stk[sp] = keep[s]; stl[sp] = keepl[s]; ++sp; }
    }
  }
  return kWalkDone;
}

// Per-query context shared by the two far kernels.
template <int DP>
struct FarQuery {
  uint32_t p, id;
  uint32_t base;   // output index of the instance's point 0 (ids - base = local ids)
  uint32_t root;   // the instance's subtree, kNoNode for a single point
  unsigned long long K;
  Pt<DP> xq;
  __device__ __forceinline__ void load(uint32_t pos, const float* __restrict__ spts,
                                       const unsigned long long* __restrict__ scode,
                                       const unsigned long long* __restrict__ skey,
                                       const ClassView& cv, const uint32_t* __restrict__ roots,
                                       int S, int ib) {
    p = pos;
    K = skey[p];
    id = key_id(K);
    xq = load_pt<DP>(spts, p);
    uint32_t inst = key_inst(scode[p], S, ib);
    if (inst >= cv.ninst) inst = 0;
    base = (uint32_t)cv.instance(inst).out;
    root = roots[inst];
  }
};

// Far queries, first round: one thread per query, a depth-first search with
// an expansion budget.  Most queries finish within it (they expand a few dozen
// nodes); the others are passed to the second round with the best distance
// found so far, which bounds their search there.
template <int DP, bool F64>
__global__ void __launch_bounds__(kFarThreads)
k_dep_far(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
          const unsigned long long* __restrict__ skey, ClassView cv,
          const CutGeom* __restrict__ cuts, const Node* __restrict__ nodes,
          const float* __restrict__ nbox, const uint32_t* __restrict__ roots, FarQueue q,
          int32_t* __restrict__ lambda, double* __restrict__ delta, Counters* ctr) {
  const uint32_t qn = ctr->queue_n;
  const uint32_t n = cv.N;
  const int S = cv.cls->S, ib = cv.cls->ib;
  // the band depends only on DP, the same for every instance of the class
  const float bmul = cuts[0].band_mul, badd = cuts[0].band_add;
  const uint32_t lanemask_lt = (1u << (threadIdx.x & 31)) - 1u;
  unsigned long long rescans = 0, expanded_sum = 0;
  uint32_t expanded_max = 0;
  bool bad = false;
  const uint32_t qn_pad = (qn + 31) & ~31u;  // whole warps, for the ballot below
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < qn_pad; e += gridDim.x * blockDim.x) {
    bool pass_on = false;
    double s_next = INFINITY;
    uint32_t expanded = 0;
    FarQuery<DP> fq;
    if (e < qn) {
      fq.load(q.pos[e], spts, scode, skey, cv, roots, S, ib);
      if (fq.root == kNoNode) {
        lambda[fq.id] = -1;
        delta[fq.id] = INFINITY;
      } else if constexpr (F64) {
        Best<double> best;
        best.init();
        const double s_init = q.s1d[e];
        const int r = tree_walk_from<DP>(
            nodes, nbox, n, skey, fq.K, fq.xq, fq.root, kFarBudget, expanded,
            [&](float lbs) { return (double)lbs > fmin(best.s1, s_init); },
            [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
              best.add(dist64<DP>(fq.xq, x), key_id(kt), t);
            });
        bad |= r == kWalkBad;
        if (r == kWalkBudget) {
          pass_on = true;
          s_next = fmin(best.s1, s_init);
        } else if (best.t1 == 0xffffffffu) {
          lambda[fq.id] = -1;
          delta[fq.id] = INFINITY;
        } else {
          lambda[fq.id] = (int32_t)(best.o1 - fq.base);
          delta[fq.id] = sqrt(best.s1);
        }
      } else {
        Best<float> best;
        best.init();
        const float s_init = q.s1[e];
        const int r = tree_walk_from<DP>(
            nodes, nbox, n, skey, fq.K, fq.xq, fq.root, kFarBudget, expanded,
            [&](float lbs) { return beyond(lbs, band_of(fminf(best.s1, s_init), bmul, badd)); },
            [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
              best.add(dist32<DP>(fq.xq, x), key_id(kt), t);
            });
        bad |= r == kWalkBad;
        if (r == kWalkBudget) {
          pass_on = true;
          s_next = fminf(best.s1, s_init);
        } else if (best.t1 == 0xffffffffu) {
          lambda[fq.id] = -1;
          delta[fq.id] = INFINITY;
        } else {
          const float b = band_of(best.s1, bmul, badd);
          Exact ex;
          ex.init();
          if (best.s2 <= b) {  // near tie: re-rank the band in binary64
            ++rescans;
            uint32_t more = 0;
            bad |= tree_walk_from<DP>(
                       nodes, nbox, n, skey, fq.K, fq.xq, fq.root, 0xffffffffu, more,
                       [&](float lbs) { return beyond(lbs, b); },
                       [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
                         if (dist32<DP>(fq.xq, x) <= b) ex.add(dist64<DP>(fq.xq, x), key_id(kt));
                       }) != kWalkDone;
            expanded += more;
          } else {
            ex.add(dist64<DP>(fq.xq, load_pt<DP>(spts, best.t1)), best.o1);
          }
          lambda[fq.id] = (int32_t)(ex.o - fq.base);
          delta[fq.id] = sqrt(ex.s);
        }
      }
    }
    expanded_sum += expanded;
    expanded_max = max(expanded_max, expanded);
    const unsigned pm = __ballot_sync(kFull, pass_on);
    uint32_t base = 0;
    if ((threadIdx.x & 31) == 0 && pm) base = atomicAdd(&ctr->queue2_n, (unsigned)__popc(pm));
    base = __shfl_sync(kFull, base, 0);
    if (pass_on) {
      const uint32_t slot = base + __popc(pm & lanemask_lt);
      q.pos2[slot] = fq.p;
      if constexpr (F64) q.s1d2[slot] = s_next;
      else q.s1_2[slot] = (float)s_next;
    }
  }
  if (bad) set_status(cv.cls->status, kStatusStack);
  for (int o = 16; o > 0; o >>= 1) {
    rescans += __shfl_xor_sync(kFull, rescans, o);
    expanded_sum += __shfl_xor_sync(kFull, expanded_sum, o);
    expanded_max = max(expanded_max, __shfl_xor_sync(kFull, expanded_max, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (rescans) atomicAdd(&ctr->exact_rescans, rescans);
    if (expanded_sum) atomicAdd(&ctr->far_nodes, expanded_sum);
    if (expanded_max) atomicMax(&ctr->far_nodes_max, expanded_max);
  }
}

// Far queries, second round: the queries that exceeded the first round's
// budget, one warp per query.  The search restarts at the root with the
// first round's best as its bound, so the warp can expand 32 nodes per step
// (one per lane) without wandering: every round pops up to 32 entries from
// the warp's shared stack, each lane expands its node, and the survivors are
// pushed with a warp prefix sum.  Children that do not fit on the stack are
// searched by their lane alone.
template <int DP, bool F64>
__global__ void __launch_bounds__(kFarThreads)
k_dep_far_wide(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
               const unsigned long long* __restrict__ skey, ClassView cv,
               const CutGeom* __restrict__ cuts, const Node* __restrict__ nodes,
               const float* __restrict__ nbox, const uint32_t* __restrict__ roots, FarQueue q,
               int32_t* __restrict__ lambda, double* __restrict__ delta, Counters* ctr) {
  constexpr int kWarpsPerBlock = kFarThreads / 32;
  __shared__ uint32_t s_stk[kWarpsPerBlock][kWarpStack];
  __shared__ float s_lb[kWarpsPerBlock][kWarpStack];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t* stk = s_stk[wib];
  float* stl = s_lb[wib];
  const uint32_t qn = ctr->queue2_n;
  const uint32_t n = cv.N;
  const int S = cv.cls->S, ib = cv.cls->ib;
  const float bmul = cuts[0].band_mul, badd = cuts[0].band_add;
  unsigned long long rescans = 0, expanded_sum = 0;
  uint32_t expanded_max = 0;
  bool bad = false;
  const uint32_t nwarps = gridDim.x * kWarpsPerBlock;
  for (uint32_t e = blockIdx.x * kWarpsPerBlock + wib; e < qn; e += nwarps) {
    FarQuery<DP> fq;
    fq.load(q.pos2[e], spts, scode, skey, cv, roots, S, ib);
    uint32_t expanded = 0;

    auto search = [&](auto refresh, auto prune, auto visit) {
      if (lane == 0) {
        stk[0] = fq.root;
        stl[0] = 0.f;
      }
      int sp = 1;
      __syncwarp();
      while (sp > 0) {
        refresh();
        const int take = sp < 32 ? sp : 32;
        const int base = sp - take;
        uint32_t keep[2];
        float keepl[2];
        int nk = 0;
        if (lane < take) {
          const uint32_t ni = stk[base + lane];
          const float lbn = stl[base + lane];
          if (!prune(lbn)) {
            if (ni + 1 >= n) {
              bad = true;
            } else {
              ++expanded;
              const ChildRec<DP> r = load_rec<DP>(nbox, ni);
#pragma unroll
              for (int s = 0; s < 2; ++s) {
                const uint32_t c = r.child[s];
                if (r.key[s] <= fq.K) continue;  // nothing of higher key below
                if (c & kLeafBit) {
                  if ((c & ~kLeafBit) >= n) {
                    bad = true;
                    continue;
                  }
                  visit(c & ~kLeafBit, r.key[s], rec_point<DP>(r, s));
                } else {
                  const float l = rec_lb2<DP>(r, s, fq.xq);
                  if (prune(l)) continue;
                  keep[nk] = c;
                  keepl[nk] = l;
                  ++nk;
                }
              }
              if (nk == 2 && keepl[0] < keepl[1]) {  // farther first: nearer is popped sooner
                const uint32_t tc = keep[0]; keep[0] = keep[1]; keep[1] = tc;
                const float tl = keepl[0]; keepl[0] = keepl[1]; keepl[1] = tl;
              }
            }
          }
        }
        uint32_t incl = (uint32_t)nk;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += t;
        }
        const int total = (int)__shfl_sync(kFull, incl, 31);
        const int pos = base + (int)incl - nk;
        __syncwarp();
        for (int s = 0; s < nk; ++s) {
          if (pos + s < kWarpStack) {
            stk[pos + s] = keep[s];
            stl[pos + s] = keepl[s];
          } else {  // no room: this lane searches the subtree alone
            bad |= tree_walk_from<DP>(nodes, nbox, n, skey, fq.K, fq.xq, keep[s], 0xffffffffu,
                                      expanded, prune, visit) != kWalkDone;
          }
        }
        sp = min(base + total, kWarpStack);
        __syncwarp();
      }
    };

    if constexpr (F64) {
      Best<double> best;
      best.init();
      const double s_init = q.s1d2[e];
      double wbest = s_init;  // the warp's best, refreshed every round
      search(
          [&] {
            double m = best.s1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(kFull, m, o));
            wbest = fmin(m, s_init);
          },
          [&](float lbs) { return (double)lbs > fmin(best.s1, wbest); },
          [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
            best.add(dist64<DP>(fq.xq, x), key_id(kt), t);
          });
      best.merge_warp();
      if (lane == 0) {
        if (best.t1 == 0xffffffffu) {
          lambda[fq.id] = -1;
          delta[fq.id] = INFINITY;
        } else {
          lambda[fq.id] = (int32_t)(best.o1 - fq.base);
          delta[fq.id] = sqrt(best.s1);
        }
      }
    } else {
      Best<float> best;
      best.init();
      const float s_init = q.s1_2[e];
      float wbest = s_init;  // the warp's best, refreshed every round
      search(
          [&] {
            float m = best.s1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(kFull, m, o));
            wbest = fminf(m, s_init);
          },
          [&](float lbs) { return beyond(lbs, band_of(fminf(best.s1, wbest), bmul, badd)); },
          [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
            best.add(dist32<DP>(fq.xq, x), key_id(kt), t);
          });
      best.merge_warp();
      if (best.t1 == 0xffffffffu) {
        if (lane == 0) {
          lambda[fq.id] = -1;
          delta[fq.id] = INFINITY;
        }
      } else {
        const float b = band_of(best.s1, bmul, badd);
        Exact ex;
        ex.init();
        if (best.s2 <= b) {  // near tie: re-rank the band in binary64
          ++rescans;
          search([] {}, [&](float lbs) { return beyond(lbs, b); },
                 [&](uint32_t t, unsigned long long kt, const Pt<DP>& x) {
                   if (dist32<DP>(fq.xq, x) <= b) ex.add(dist64<DP>(fq.xq, x), key_id(kt));
                 });
          ex.merge_warp();
        } else if (lane == 0) {
          ex.add(dist64<DP>(fq.xq, load_pt<DP>(spts, best.t1)), best.o1);
        }
        if (lane == 0) {
          lambda[fq.id] = (int32_t)(ex.o - fq.base);
          delta[fq.id] = sqrt(ex.s);
        }
      }
    }
    expanded_sum += expanded;
    uint32_t qexp = expanded;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qexp += __shfl_xor_sync(kFull, qexp, o);
    expanded_max = max(expanded_max, qexp);
  }
  if (__any_sync(kFull, bad) && lane == 0) set_status(cv.cls->status, kStatusStack);
  for (int o = 16; o > 0; o >>= 1) expanded_sum += __shfl_xor_sync(kFull, expanded_sum, o);
  if (lane == 0) {
    if (rescans) atomicAdd(&ctr->exact_rescans, rescans);
    if (expanded_sum) atomicAdd(&ctr->far_nodes, expanded_sum);
    if (expanded_max) atomicMax(&ctr->far_nodes_max, expanded_max);
  }
}

__global__ void k_far_count(Counters* ctr) {
  ctr->far_queries += ctr->queue_n;
  ctr->far_wide_queries += ctr->queue2_n;
}


inline unsigned grid_for(uint64_t items, int per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, int G>
void near_dg(bool fp64, int layout, const float* spts, const unsigned long long* scode,
             const unsigned long long* skey, const ClassView& cv, int32_t rho_skip,
             const void* pts, int dtype, const CutGeom* cuts, const HashInfo* hi,
             const unsigned long long* hkeys, const uint2* hvals, int32_t* lambda, double* delta,
             FarQueue q, Counters* ctr, int seg_cells, cudaStream_t st) {
  const unsigned grid = grid_for(cv.nchunk, kNearWarps, sm_count() * 64u);
  if (layout == kLayoutSegment) {
    if (fp64)
      k_dep_near_seg<DP, G, true><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                                 dtype, cuts, hi, hkeys, hvals, lambda,
                                                                 delta, q, ctr, seg_cells);
    else
      k_dep_near_seg<DP, G, false><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                                  dtype, cuts, hi, hkeys, hvals, lambda,
                                                                  delta, q, ctr, seg_cells);
  } else {
    if (fp64)
      k_dep_near<DP, G, true><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                             dtype, cuts, hi, hkeys, hvals, lambda,
                                                             delta, q, ctr);
    else
      k_dep_near<DP, G, false><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                              dtype, cuts, hi, hkeys, hvals, lambda,
                                                              delta, q, ctr);
  }
}

template <int DP>
void far_dp(bool fp64, const float* spts, const unsigned long long* scode,
            const unsigned long long* skey, const ClassView& cv, const CutGeom* cuts,
            const Node* nodes, const float* nbox, const uint32_t* root, FarQueue q,
            int32_t* lambda, double* delta, Counters* ctr, cudaStream_t st) {
  // the queue length is known only on the device: launch enough threads for
  // a full SM load and let them stride over it
  const unsigned grid = grid_for(cv.N, kFarThreads, sm_count() * 8u);
  const unsigned grid2 = grid_for(cv.N, kFarThreads / 32, sm_count() * 16u);
  if (fp64) {
    k_dep_far<DP, true><<<grid, kFarThreads, 0, st>>>(spts, scode, skey, cv, cuts, nodes, nbox,
                                                      root, q, lambda, delta, ctr);
    k_dep_far_wide<DP, true><<<grid2, kFarThreads, 0, st>>>(spts, scode, skey, cv, cuts, nodes,
                                                            nbox, root, q, lambda, delta, ctr);
  } else {
    k_dep_far<DP, false><<<grid, kFarThreads, 0, st>>>(spts, scode, skey, cv, cuts, nodes, nbox,
                                                       root, q, lambda, delta, ctr);
    k_dep_far_wide<DP, false><<<grid2, kFarThreads, 0, st>>>(spts, scode, skey, cv, cuts, nodes,
                                                             nbox, root, q, lambda, delta, ctr);
  }
}

}  // namespace

void launch_dep_near(int dp, int g, bool fp64, int layout, const float* spts,
                     const unsigned long long* scode, const unsigned long long* skey,
                     const ClassView& cv, int32_t rho_skip, const void* pts, int dtype,
                     const CutGeom* cuts, const HashInfo* hi, const unsigned long long* hkeys,
                     const uint2* hvals, int32_t* lambda, double* delta, FarQueue q, Counters* ctr,
                     cudaStream_t st, int seg_cells) {
  if (cv.N == 0) return;
  cudaMemsetAsync(&ctr->queue_n, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(&ctr->queue2_n, 0, sizeof(unsigned int), st);
  if (layout == kLayoutCell) {
    launch_dep_near_cell(dp, g, fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys,
                         hvals, lambda, delta, q, ctr, st);
    return;  // counted there
  }
  if (layout == kLayoutTree) {
    k_near_to_far<<<grid_for((uint64_t)cv.nchunk * 32u, 256, sm_count() * 16u), 256, 0, st>>>(
        skey, cv, cuts, rho_skip, lambda, delta, q, ctr);
  } else if (g == 1) near_dg<2, 1>(fp64, layout, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, seg_cells, st);
  else if (g == 2) near_dg<2, 2>(fp64, layout, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, seg_cells, st);
  else if (g == 3) near_dg<4, 3>(fp64, layout, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, seg_cells, st);
  else if (dp == 4) near_dg<4, 4>(fp64, layout, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, seg_cells, st);
  else near_dg<8, 4>(fp64, layout, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, seg_cells, st);
  count_launches(1);
}

void launch_dep_far(int dp, bool fp64, const float* spts, const unsigned long long* scode,
                    const unsigned long long* skey, const ClassView& cv, const CutGeom* cuts,
                    const Node* nodes, const float* nbox, const uint32_t* root, FarQueue q,
                    int32_t* lambda, double* delta, Counters* ctr, cudaStream_t st) {
  if (cv.N == 0) return;
  if (dp == 2) far_dp<2>(fp64, spts, scode, skey, cv, cuts, nodes, nbox, root, q, lambda, delta, ctr, st);
  else if (dp == 4) far_dp<4>(fp64, spts, scode, skey, cv, cuts, nodes, nbox, root, q, lambda, delta, ctr, st);
  else far_dp<8>(fp64, spts, scode, skey, cv, cuts, nodes, nbox, root, q, lambda, delta, ctr, st);
  k_far_count<<<1, 1, 0, st>>>(ctr);
  count_launches(3);
}

}  // namespace dpc
