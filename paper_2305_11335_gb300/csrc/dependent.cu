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

// Coordinates of point `id` from the caller's input (the same float values the
// sorted copy holds: int32 inputs are exact in float32 by the range check).
template <int DP>
__device__ __forceinline__ Pt<DP> input_pt(const void* __restrict__ pts, int dtype, int d, uint32_t id) {
  Pt<DP> p;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
    float v = 0.f;
    if (a < d) {
      const size_t e = (size_t)id * d + a;
      v = dtype == 0 ? (float)__ldg((const int32_t*)pts + e) : __ldg((const float*)pts + e);
    }
    p.x[a] = v;
  }
  return p;
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kNearThreads)
k_dep_near(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
           const unsigned long long* __restrict__ skey, uint32_t n, int32_t rho_skip,
           const void* __restrict__ pts, int dtype, int d,
           const GridGeom* __restrict__ geom, const CutGeom* __restrict__ cut,
           const unsigned long long* __restrict__ hkeys, const uint2* __restrict__ hvals,
           int32_t* __restrict__ lambda, double* __restrict__ delta, FarQueue q, Counters* ctr) {
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
  const float f2lo = geom->f2 * (1.f - 1e-5f);
  const double inv_f = geom->inv_f;
  double org[G];
#pragma unroll
  for (int a = 0; a < G; ++a) org[a] = geom->org[a];
  const int k = cut->k;
  const float cell_fine = (float)(1u << cut->k);
  const int R = cut->R;
  const int shift = G * k;
  const int cmax = (1 << (geom->B - k)) - 1;
  const uint32_t hmask = cut->hmask;
  const float bmul = cut->band_mul, badd = cut->band_add;
  const float far32 = cut->far32;
  const double far64 = cut->far64;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  const uint32_t nchunk = (n + 31) / 32;
  for (uint32_t ch = blockIdx.x * kNearWarps + wib; ch < nchunk; ch += gridDim.x * kNearWarps) {
    const uint32_t p = ch * 32 + lane;
    const bool valid = p < n;
    Pt<DP> me;
#pragma unroll
    for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
    unsigned long long K = ~0ull;
    if (valid) {
      me = load_pt<DP>(spts, p);
      K = skey[p];
    }
    const unsigned long long mycell = valid ? (scode[p] >> shift) : ~0ull;
    uint32_t c0[G];
    unmorton<G>(valid ? mycell : 0ull, c0);
    const bool skip = valid && (int32_t)(K >> 32) < rho_skip;
    const int nvalid = (int)min(32u, n - ch * 32);
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
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, n, lane, rt);
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
          lambda[id] = (int32_t)acc64.o;
          delta[id] = sqrt(acc64.s);
        }
      } else if (acc.o1 != 0xffffffffu) {
        s1 = acc.s1;
        const float bnd = band_of(s1, bmul, badd);
        settled = bnd < far32 && acc.s2 > bnd;
        if (settled) {
          lambda[id] = (int32_t)acc.o1;
          delta[id] = sqrt(dist64<DP>(me, input_pt<DP>(pts, dtype, d, acc.o1)));
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

// ---------------------------------------------------------------------------
// far phase: depth-first priority search of the radix tree

template <int G>
__device__ __forceinline__ float node_lb2(const Node& nd, int nbits, const float* u) {
  const int nb = nbits - (int)nd.plen;  // free low bits of the code
  uint32_t c[G];
  unmorton<G>(nd.code, c);
  float lb2 = 0.f;
#pragma unroll
  for (int a = 0; a < G; ++a) {
    const int fa = nb > a ? (nb - a + G - 1) / G : 0;
    const uint32_t lo = (c[a] >> fa) << fa;
    const float l = lb_axis((float)lo, (float)lo + (float)((1u << fa) - 1u), u[a]);
    lb2 = fmaf(l, l, lb2);
  }
  return lb2;
}

// Visit every candidate (leaf with key > K) not excluded by `prune`; calls
// visit(t, kt) for each.  prune(lbs) says whether a region whose squared
// distance is at least lbs can be skipped.  Returns false if the tree is
// malformed or the stack would overflow (neither happens for a tree built by
// tree.cu: its depth is at most 64 + 32).
template <int DP, int G, typename Prune, typename Visit>
__device__ __forceinline__ bool tree_walk(const Node* __restrict__ nodes, uint32_t n, int nbits,
                                          const unsigned long long* __restrict__ skey,
                                          unsigned long long K, const float* u, float f2lo,
                                          Prune prune, Visit visit) {
  uint32_t stk[kStack];
  float stl[kStack];
  int sp = 0;
  if (n == 1) {
    const unsigned long long kt = skey[0];
    if (kt > K) visit(0u, kt);
    return true;
  }
  stk[sp] = 0u;
  stl[sp] = 0.f;
  ++sp;
  while (sp > 0) {
    --sp;
    const uint32_t ni = stk[sp];
    if (prune(stl[sp])) continue;
    if (ni + 1 >= n) return false;
    const uint32_t ch[2] = {nodes[ni].left, nodes[ni].right};
    uint32_t keep[2];
    float keepl[2];
    int nk = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t c = ch[s];
      if (c & kLeafBit) {
        const uint32_t t = c & ~kLeafBit;
        if (t >= n) return false;
        const unsigned long long kt = skey[t];
        if (kt > K) visit(t, kt);
      } else {
        const Node nd = nodes[c];
        if (nd.maxkey <= K) continue;
        const float lbs = node_lb2<G>(nd, nbits, u) * f2lo;
        if (prune(lbs)) continue;
        keep[nk] = c;
        keepl[nk] = lbs;
        ++nk;
      }
    }
    if (sp + nk > kStack) return false;
    if (nk == 2 && keepl[0] < keepl[1]) {  // push the farther child first
      stk[sp] = keep[1]; stl[sp] = keepl[1]; ++sp;
      stk[sp] = keep[0]; stl[sp] = keepl[0]; ++sp;
    } else {
      for (int s = 0; s < nk; ++s) { stk[sp] = keep[s]; stl[sp] = keepl[s]; ++sp; }
    }
  }
  return true;
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kFarThreads)
k_dep_far(const float* __restrict__ spts, const unsigned long long* __restrict__ skey, uint32_t n,
          const GridGeom* __restrict__ geom, const CutGeom* __restrict__ cut,
          const Node* __restrict__ nodes, FarQueue q, int32_t* __restrict__ lambda,
          double* __restrict__ delta, Counters* ctr) {
  const uint32_t qn = ctr->queue_n;
  const int nbits = geom->nbits;
  const float bmul = cut->band_mul, badd = cut->band_add;
  const float f2lo = geom->f2 * (1.f - 1e-5f);
  const double inv_f = geom->inv_f;
  double org[G];
#pragma unroll
  for (int a = 0; a < G; ++a) org[a] = geom->org[a];
  unsigned long long rescans = 0;
  bool overflow = false;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < qn; e += gridDim.x * blockDim.x) {
    const uint32_t p = q.pos[e];
    const unsigned long long K = skey[p];
    const uint32_t id = key_id(K);
    const Pt<DP> xq = load_pt<DP>(spts, p);
    float u[G];
#pragma unroll
    for (int a = 0; a < G; ++a) u[a] = (float)(((double)xq.x[a] - org[a]) * inv_f);

    if constexpr (F64) {
      Best<double> best;
      best.init();
      const double s_init = q.s1d[e];
      overflow |= !tree_walk<DP, G>(
          nodes, n, nbits, skey, K, u, f2lo,
          [&](float lbs) { return (double)lbs > fmin(best.s1, s_init); },
          [&](uint32_t t, unsigned long long kt) {
            best.add(dist64<DP>(xq, load_pt<DP>(spts, t)), key_id(kt), t);
          });
      if (best.t1 == 0xffffffffu) {
        lambda[id] = -1;
        delta[id] = INFINITY;
      } else {
        lambda[id] = (int32_t)best.o1;
        delta[id] = sqrt(best.s1);
      }
    } else {
      Best<float> best;
      best.init();
      const float s_init = q.s1[e];
      overflow |= !tree_walk<DP, G>(
          nodes, n, nbits, skey, K, u, f2lo,
          [&](float lbs) { return beyond(lbs, band_of(fminf(best.s1, s_init), bmul, badd)); },
          [&](uint32_t t, unsigned long long kt) {
            best.add(dist32<DP>(xq, load_pt<DP>(spts, t)), key_id(kt), t);
          });
      if (best.t1 == 0xffffffffu) {
        lambda[id] = -1;
        delta[id] = INFINITY;
        continue;
      }
      const float b = band_of(best.s1, bmul, badd);
      Exact ex;
      ex.init();
      if (best.s2 <= b) {
        ++rescans;
        overflow |= !tree_walk<DP, G>(
            nodes, n, nbits, skey, K, u, f2lo, [&](float lbs) { return beyond(lbs, b); },
            [&](uint32_t t, unsigned long long kt) {
              const Pt<DP> x = load_pt<DP>(spts, t);
              if (dist32<DP>(xq, x) <= b) ex.add(dist64<DP>(xq, x), key_id(kt));
            });
      } else {
        ex.add(dist64<DP>(xq, load_pt<DP>(spts, best.t1)), best.o1);
      }
      lambda[id] = (int32_t)ex.o;
      delta[id] = sqrt(ex.s);
    }
  }
  if (overflow) set_status(geom->status, kStatusStack);
  for (int o = 16; o > 0; o >>= 1) rescans += __shfl_xor_sync(kFull, rescans, o);
  if ((threadIdx.x & 31) == 0 && rescans) atomicAdd(&ctr->exact_rescans, rescans);
}

__global__ void k_far_count(Counters* ctr) { ctr->far_queries += ctr->queue_n; }

inline unsigned grid_for(uint64_t items, int per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, int G>
void near_dg(bool fp64, const float* spts, const unsigned long long* scode,
             const unsigned long long* skey, uint32_t n, int32_t rho_skip, const void* pts,
             int dtype, int d, const GridGeom* geom,
             const CutGeom* cut, const unsigned long long* hkeys, const uint2* hvals,
             int32_t* lambda, double* delta, FarQueue q, Counters* ctr, cudaStream_t st) {
  const unsigned grid = grid_for((n + 31) / 32, kNearWarps, 152u * 64u);
  if (fp64)
    k_dep_near<DP, G, true><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, n, rho_skip, pts, dtype,
                                                           d, geom, cut, hkeys, hvals, lambda, delta,
                                                           q, ctr);
  else
    k_dep_near<DP, G, false><<<grid, kNearThreads, 0, st>>>(spts, scode, skey, n, rho_skip, pts,
                                                            dtype, d, geom, cut, hkeys, hvals, lambda,
                                                            delta, q, ctr);
}

template <int DP, int G>
void far_dg(bool fp64, const float* spts, const unsigned long long* skey, uint32_t n,
            const GridGeom* geom, const CutGeom* cut, const Node* nodes, FarQueue q,
            int32_t* lambda, double* delta, Counters* ctr, uint32_t qcap, cudaStream_t st) {
  // the queue length is known only on the device: launch enough threads for
  // a full SM load and let them stride over it
  const unsigned grid = grid_for(qcap, kFarThreads, 152u * 8u);
  if (fp64)
    k_dep_far<DP, G, true><<<grid, kFarThreads, 0, st>>>(spts, skey, n, geom, cut, nodes, q, lambda,
                                                         delta, ctr);
  else
    k_dep_far<DP, G, false><<<grid, kFarThreads, 0, st>>>(spts, skey, n, geom, cut, nodes, q, lambda,
                                                          delta, ctr);
}

}  // namespace

void launch_dep_near(int dp, int g, bool fp64, const float* spts, const unsigned long long* scode,
                     const unsigned long long* skey, uint32_t n, int32_t rho_skip, const void* pts,
                     int dtype, int d, const GridGeom* geom, const CutGeom* cut, const unsigned long long* hkeys,
                     const uint2* hvals, int32_t* lambda, double* delta, FarQueue q,
                     Counters* ctr, cudaStream_t st) {
  if (n == 0) return;
  cudaMemsetAsync(&ctr->queue_n, 0, sizeof(unsigned int), st);
  if (g == 1) near_dg<2, 1>(fp64, spts, scode, skey, n, rho_skip, pts, dtype, d, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (g == 2) near_dg<2, 2>(fp64, spts, scode, skey, n, rho_skip, pts, dtype, d, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (dp == 4) near_dg<4, 3>(fp64, spts, scode, skey, n, rho_skip, pts, dtype, d, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else near_dg<8, 3>(fp64, spts, scode, skey, n, rho_skip, pts, dtype, d, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  count_launches(1);
}

void launch_dep_far(int dp, int g, bool fp64, const float* spts, const unsigned long long* skey,
                    uint32_t n, const GridGeom* geom, const CutGeom* cut, const Node* nodes,
                    FarQueue q, int32_t* lambda, double* delta, Counters* ctr, uint32_t qcap,
                    cudaStream_t st) {
  if (n == 0) return;
  if (g == 1) far_dg<2, 1>(fp64, spts, skey, n, geom, cut, nodes, q, lambda, delta, ctr, qcap, st);
  else if (g == 2) far_dg<2, 2>(fp64, spts, skey, n, geom, cut, nodes, q, lambda, delta, ctr, qcap, st);
  else if (dp == 4) far_dg<4, 3>(fp64, spts, skey, n, geom, cut, nodes, q, lambda, delta, ctr, qcap, st);
  else far_dg<8, 3>(fp64, spts, skey, n, geom, cut, nodes, q, lambda, delta, ctr, qcap, st);
  k_far_count<<<1, 1, 0, st>>>(ctr);
  count_launches(2);
}

}  // namespace dpc
