// dependent.cu -- lambda_i (the nearest point of higher order) and
// delta_i = D(x_i, lambda_i) (Definitions 2-3).
//
// The paper runs one priority nearest-neighbour query per point in parallel
// (Algorithm 1) on a priority search kd-tree.  Here each query runs in two
// phases:
//   near  scan the (2R+1)^g grid block around the point (the same cells the
//         density used).  If the best candidate is closer than anything
//         outside the block can be, the query is settled; this holds for most
//         points, since a point's dependent point is usually within d_cut.
//   far   the remaining queries (local density maxima, isolated points) walk
//         the radix tree (tree.cu) depth first, nearer child first, skipping
//         subtrees whose largest key is not above the query's key or whose
//         box is farther than the best candidate so far (Section 4.1.2).
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

#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 128;
constexpr int kStack = 128;

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

// Running minimum of (s, id) plus the second smallest s.
template <typename S>
struct Best {
  S s1, s2;
  uint32_t o1;   // id of the best
  uint32_t t1;   // sorted position of the best
  __device__ __forceinline__ void init(S inf) {
    s1 = inf;
    s2 = inf;
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

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads)
k_dep_near(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
           const unsigned long long* __restrict__ skey, uint32_t n, int32_t rho_skip,
           const GridGeom* __restrict__ geom, const CutGeom* __restrict__ cut,
           const unsigned long long* __restrict__ hkeys, const uint2* __restrict__ hvals,
           int32_t* __restrict__ lambda, double* __restrict__ delta, FarQueue q, Counters* ctr) {
  const int k = cut->k;
  const int R = cut->R;
  const int W = 2 * R + 1;
  const int shift = G * k;
  const int cmax = (1 << (geom->B - k)) - 1;
  const float cell_fine = (float)(1u << k);
  const uint32_t hmask = cut->hmask;
  const float bmul = cut->band_mul, badd = cut->band_add;
  const float far32 = cut->far32;
  const double far64 = cut->far64;
  // fine-unit squared lower bound -> conservative float lower bound of s
  const float f2lo = geom->f2 * (1.f - 1e-5f);
  const double inv_f = geom->inv_f;
  double org[G];
#pragma unroll
  for (int a = 0; a < G; ++a) org[a] = geom->org[a];
  int ncell = 1;
  for (int a = 0; a < G; ++a) ncell *= W;

  unsigned long long rescans = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned long long K = skey[p];
    const uint32_t id = key_id(K);
    if ((int32_t)(K >> 32) < rho_skip) {
      lambda[id] = -1;
      delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
      continue;
    }
    const Pt<DP> xq = load_pt<DP>(spts, p);
    float u[G];
#pragma unroll
    for (int a = 0; a < G; ++a) u[a] = (float)(((double)xq.x[a] - org[a]) * inv_f);
    uint32_t c0[G];
    unmorton<G>(scode[p] >> shift, c0);

    using S = typename std::conditional<F64, double, float>::type;
    Best<S> best;
    best.init((S)INFINITY);
    for (int o = 0; o < ncell; ++o) {
      int rem = o;
      uint32_t c[G];
      float lb2 = 0.f;
      bool inside = true;
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int off = rem % W - R;
        rem /= W;
        const int ca = (int)c0[a] + off;
        inside &= (ca >= 0) & (ca <= cmax);
        c[a] = (uint32_t)ca;
        const float lo = (float)ca * cell_fine;
        const float l = lb_axis(lo, lo + cell_fine - 1.f, u[a]);
        lb2 = fmaf(l, l, lb2);
      }
      if (!inside) continue;
      const float lbs = lb2 * f2lo;
      if constexpr (F64) {
        if ((double)lbs > best.s1) continue;
      } else {
        if (beyond(lbs, band_of(best.s1, bmul, badd))) continue;
      }
      const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, morton<G>(c)), n);
      for (uint32_t t = run.x; t < run.y; ++t) {
        const unsigned long long kt = skey[t];
        if (kt <= K) continue;
        const Pt<DP> x = load_pt<DP>(spts, t);
        if constexpr (F64) best.add(dist64<DP>(xq, x), key_id(kt), t);
        else best.add(dist32<DP>(xq, x), key_id(kt), t);
      }
    }

    bool settled;
    if constexpr (F64) {
      settled = best.t1 != 0xffffffffu && best.s1 < far64;
      if (settled) {
        lambda[id] = (int32_t)best.o1;
        delta[id] = sqrt(best.s1);
      }
    } else {
      const float b = band_of(best.s1, bmul, badd);
      settled = best.t1 != 0xffffffffu && b < far32;
      if (settled) {
        Exact ex;
        ex.init();
        if (best.s2 <= b) {
          // ambiguous: re-rank every candidate inside the band in binary64
          ++rescans;
          for (int o = 0; o < ncell; ++o) {
            int rem = o;
            uint32_t c[G];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < G; ++a) {
              const int ca = (int)c0[a] + rem % W - R;
              rem /= W;
              inside &= (ca >= 0) & (ca <= cmax);
              c[a] = (uint32_t)ca;
            }
            if (!inside) continue;
            const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, morton<G>(c)), n);
            for (uint32_t t = run.x; t < run.y; ++t) {
              const unsigned long long kt = skey[t];
              if (kt <= K) continue;
              const Pt<DP> x = load_pt<DP>(spts, t);
              if (dist32<DP>(xq, x) <= b) ex.add(dist64<DP>(xq, x), key_id(kt));
            }
          }
        } else {
          ex.add(dist64<DP>(xq, load_pt<DP>(spts, best.t1)), best.o1);
        }
        lambda[id] = (int32_t)ex.o;
        delta[id] = sqrt(ex.s);
      }
    }
    if (!settled) {
      const uint32_t e = atomicAdd(&ctr->queue_n, 1u);
      q.pos[e] = p;
      if constexpr (F64) q.s1d[e] = best.s1;
      else q.s1[e] = best.s1;
    }
  }
  if constexpr (!F64) {
    for (int o = 16; o > 0; o >>= 1) rescans += __shfl_xor_sync(0xffffffffu, rescans, o);
    if ((threadIdx.x & 31) == 0 && rescans) atomicAdd(&ctr->exact_rescans, rescans);
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
// distance is at least lbs can be skipped.
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
    if (ni + 1 >= n) return false;  // not an internal node: corrupted tree
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
__global__ void __launch_bounds__(kThreads)
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
      best.init(INFINITY);
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
      best.init(INFINITY);
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
  for (int o = 16; o > 0; o >>= 1) rescans += __shfl_xor_sync(0xffffffffu, rescans, o);
  if ((threadIdx.x & 31) == 0 && rescans) atomicAdd(&ctr->exact_rescans, rescans);
}

__global__ void k_far_count(Counters* ctr) { ctr->far_queries += ctr->queue_n; }

inline unsigned grid_for(uint64_t n, unsigned cap) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, int G>
void near_dg(bool fp64, const float* spts, const unsigned long long* scode,
             const unsigned long long* skey, uint32_t n, int32_t rho_skip, const GridGeom* geom,
             const CutGeom* cut, const unsigned long long* hkeys, const uint2* hvals,
             int32_t* lambda, double* delta, FarQueue q, Counters* ctr, cudaStream_t st) {
  const unsigned grid = grid_for(n, 152u * 128u);
  if (fp64)
    k_dep_near<DP, G, true><<<grid, kThreads, 0, st>>>(spts, scode, skey, n, rho_skip, geom, cut,
                                                       hkeys, hvals, lambda, delta, q, ctr);
  else
    k_dep_near<DP, G, false><<<grid, kThreads, 0, st>>>(spts, scode, skey, n, rho_skip, geom, cut,
                                                        hkeys, hvals, lambda, delta, q, ctr);
}

template <int DP, int G>
void far_dg(bool fp64, const float* spts, const unsigned long long* skey, uint32_t n,
            const GridGeom* geom, const CutGeom* cut, const Node* nodes, FarQueue q,
            int32_t* lambda, double* delta, Counters* ctr, uint32_t qcap, cudaStream_t st) {
  // the queue length is known only on the device: launch enough threads for
  // a full SM load and let them stride over it
  const unsigned grid = grid_for(qcap, 152u * 8u);
  if (fp64)
    k_dep_far<DP, G, true><<<grid, kThreads, 0, st>>>(spts, skey, n, geom, cut, nodes, q, lambda,
                                                      delta, ctr);
  else
    k_dep_far<DP, G, false><<<grid, kThreads, 0, st>>>(spts, skey, n, geom, cut, nodes, q, lambda,
                                                       delta, ctr);
}

}  // namespace

void launch_dep_near(int dp, int g, bool fp64, const float* spts, const unsigned long long* scode,
                     const unsigned long long* skey, uint32_t n, int32_t rho_skip,
                     const GridGeom* geom, const CutGeom* cut, const unsigned long long* hkeys,
                     const uint2* hvals, int32_t* lambda, double* delta, FarQueue q,
                     Counters* ctr, cudaStream_t st) {
  if (n == 0) return;
  cudaMemsetAsync(&ctr->queue_n, 0, sizeof(unsigned int), st);
  if (g == 1) near_dg<2, 1>(fp64, spts, scode, skey, n, rho_skip, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (g == 2) near_dg<2, 2>(fp64, spts, scode, skey, n, rho_skip, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (dp == 4) near_dg<4, 3>(fp64, spts, scode, skey, n, rho_skip, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
  else near_dg<8, 3>(fp64, spts, scode, skey, n, rho_skip, geom, cut, hkeys, hvals, lambda, delta, q, ctr, st);
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
