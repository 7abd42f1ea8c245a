// binning.cu -- bounding box, grid geometry, Morton codes, sorted gather and
// the occupied-cell hash of the density grid level.
//
// The paper builds a kd-tree over the points before each query step
// (Section 3.2); here the spatial index is a uniform grid whose cells are
// contiguous runs of the Morton-sorted points, built with a radix sort (the
// radix-sort primitive of Section 3.2) and an open-addressing hash of the
// occupied cells.
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(uint64_t n, int threads = kThreads, unsigned cap = sm_count() * 16u) {
  uint64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// Class and per-instance geometry reset (one thread per instance).
__global__ void k_class_init(ClassView cv, int g, int ib, int bcap, int* status) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    cv.cls->S = 0;
    cv.cls->ib = ib;
    cv.cls->bcap = bcap;
    cv.cls->status = status;
  }
  if (t >= cv.ninst) return;
  GridGeom& G = cv.geom[t];
  G.g = g;
  G.status = status;
  for (int a = 0; a < kMaxGrid; ++a) {
    G.bbox_ord[a] = 0xffffffffu;        // min accumulators
    G.bbox_ord[kMaxGrid + a] = 0u;      // max accumulators
  }
}

// Bounding box of the gridded axes of every instance, and the coordinate
// range check.  In a batch each warp takes a contiguous range of chunks and
// keeps a running box while the instance stays the same, so most instances
// see one atomic per warp and axis.
template <typename T>
__device__ __forceinline__ float bbox_value(T v, int& bad) {
  if constexpr (std::is_integral<T>::value) {
    bad |= (v > (1 << 24)) | (v < -(1 << 24));
    return (float)v;
  } else {
    const float x = (float)v;
    bad |= !(fabsf(x) <= 1.152921504606846976e18f);  // 2^60; false for NaN
    return x;
  }
}

template <typename T>
__global__ void k_bbox(const T* __restrict__ pts, ClassView cv, int g) {
  if (!cv.chunk_inst) {
    // One instance: the coordinates are one array of N*d values.  A stride
    // that is a multiple of d gives every thread one axis, the loads are
    // coalesced and four are in flight per thread; the block's box is
    // reduced in shared memory, one atomic per block and gridded axis.
    __shared__ uint32_t s_lo[kMaxGrid], s_hi[kMaxGrid];
    if (threadIdx.x < kMaxGrid) {
      s_lo[threadIdx.x] = 0xffffffffu;
      s_hi[threadIdx.x] = 0u;
    }
    __syncthreads();
    const InstDev I = cv.one;
    const uint64_t d = (uint64_t)I.d;
    const uint64_t nv = (uint64_t)cv.N * d;
    const uint64_t all = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t stride = all - all % d;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float mn = FLT_MAX, mx = -FLT_MAX;
    int bad = 0;
    if (t0 < stride) {
      const T* __restrict__ src = pts + I.coord;
      uint64_t v = t0;
      for (; v + 3 * stride < nv; v += 4 * stride) {
        T q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = src[v + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float x = bbox_value<T>(q[u], bad);
          mn = fminf(mn, x);
          mx = fmaxf(mx, x);
        }
      }
      for (; v < nv; v += stride) {
        const float x = bbox_value<T>(src[v], bad);
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
      }
      const int a = (int)(t0 % d);
      if (a < g && mn <= mx) {
        atomicMin(&s_lo[a], float_ord(mn));
        atomicMax(&s_hi[a], float_ord(mx));
      }
    }
    const int any_bad = __syncthreads_or(bad);
    if (threadIdx.x < (unsigned)g && s_lo[threadIdx.x] != 0xffffffffu) {
      atomicMin(&cv.geom[0].bbox_ord[threadIdx.x], s_lo[threadIdx.x]);
      atomicMax(&cv.geom[0].bbox_ord[kMaxGrid + threadIdx.x], s_hi[threadIdx.x]);
    }
    if (any_bad && threadIdx.x == 0) set_status(cv.cls->status, kStatusBadCoord);
    return;
  }
  const int lane = threadIdx.x & 31;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t per = (cv.nchunk + nw - 1) / nw;
  const uint32_t c0 = w * per, c1 = min(cv.nchunk, c0 + per);
  float mn[kMaxGrid], mx[kMaxGrid];
  uint32_t cur = 0xffffffffu;
  int bad = 0;
  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < kMaxGrid; ++k) {
      const uint32_t lo = __reduce_min_sync(0xffffffffu, float_ord(mn[k]));
      const uint32_t hi = __reduce_max_sync(0xffffffffu, float_ord(mx[k]));
      if (lane == 0 && k < g && ord_float(lo) <= ord_float(hi)) {
        atomicMin(&cv.geom[cur].bbox_ord[k], lo);
        atomicMax(&cv.geom[cur].bbox_ord[kMaxGrid + k], hi);
      }
    }
  };
  for (uint32_t c = c0; c < c1; ++c) {
    uint32_t i, p0, end;
    cv.chunk(c, i, p0, end);
    if (i != cur) {
      if (cur != 0xffffffffu) flush();
      cur = i;
#pragma unroll
      for (int k = 0; k < kMaxGrid; ++k) {
        mn[k] = FLT_MAX;
        mx[k] = -FLT_MAX;
      }
    }
    const InstDev I = cv.instance(i);
    const uint32_t p = p0 + lane;
    if (p < end) {
      const T* row = pts + I.coord + (size_t)(p - I.start) * I.d;
      for (int a = 0; a < I.d; ++a) {
        const float x = bbox_value<T>(row[a], bad);
        if (a < kMaxGrid) {
#pragma unroll
          for (int k = 0; k < kMaxGrid; ++k)
            if (k == a) { mn[k] = fminf(mn[k], x); mx[k] = fmaxf(mx[k], x); }
        }
      }
    }
  }
  if (cur != 0xffffffffu) flush();
  if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(cv.cls->status, kStatusBadCoord);
}

// Grid geometry of every instance from its bounding box (one thread each).
//
// Fine grid: the fine cell is 1/8 of the instance's smallest cutoff (times
// 1 + 2^-20), so the level-3 cell is just wider than d_cut and the 3^g block
// around it holds every point within d_cut with the least volume a cell grid
// allows.  At most bcap <= kMaxBits bits per axis keep fine-unit coordinates
// exact to 1/8 cell in float32 (and the sort key below 2^63); a wider bounding
// box gets a coarser fine cell instead.  A point's fine index
// c = floor((x - org) * inv_f) is within 1e-9 cells of the exact real value,
// so its real position lies in [c - 0.5, c + 1.5) fine units; every bound
// below is derived from that interval.
__global__ void k_setup_geom(ClassView cv, int ncut, const CutHost* __restrict__ hc, CutArgs args) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cv.ninst) return;
  GridGeom* geom = cv.geom + t;
  double dcmin = INFINITY;
  for (int c = 0; c < ncut; ++c) dcmin = fmin(dcmin, hc ? hc[(size_t)t * ncut + c].dc : args.h[c].dc);
  const int g = geom->g;
  const int bcap = cv.cls->bcap;
  double E = 0.0;
  for (int a = 0; a < g; ++a) {
    uint32_t lo = geom->bbox_ord[a], hi = geom->bbox_ord[kMaxGrid + a];
    double mn = 0.0, mx = 0.0;
    if (lo != 0xffffffffu) {
      mn = (double)ord_float(lo);
      mx = (double)ord_float(hi);
    }
    geom->org[a] = mn;
    E = fmax(E, mx - mn);
  }
  int B;
  double f;
  if (!(E > 0.0)) {
    B = 1;
    f = 1.0;
  } else {
    const double f_fit = dcmin * (1.0 + 0x1p-20) * 0.125;
    if (f_fit > 0.0 && E / f_fit < ldexp(1.0, bcap) * (1.0 - 0x1p-20)) {
      f = f_fit;
      B = 1;
      while (ldexp(f, B) <= E * (1.0 + 0x1p-30)) ++B;  // E / f < 2^B with margin
    } else {
      B = bcap;
      f = ldexp(E, -B) * (1.0 + 0x1p-20);
    }
  }
  geom->B = B;
  geom->f = f;
  geom->inv_f = 1.0 / f;
  geom->f2 = __double2float_rd(f * f);
  geom->nbits = g * B;
  atomicMax(&cv.cls->S, g * B);
}

// Grid level k and block radius R of one (instance, cutoff), and the bounds
// that follow from them.  Two points within d_cut differ by at most D fine
// indices on each axis, so any (k, R) with R * 2^k >= D puts every point
// within d_cut of a query in the (2R+1)^g block of level-k cells around it.
// rpref = 0: R = 1 (the 3^g block of cells at least d_cut wide) unless a
// larger R on finer cells shrinks the block side by more than 20%, which pays
// for its extra cell lookups (it happens when d_cut falls just above a
// power-of-two multiple of the fine cell, e.g. the larger cutoffs of a sweep).
// rpref > 0: the finest level whose block radius is at most rpref (the
// autotuner's choice, see api.cu).
// Points outside the (2R+1)^g block of level-k cells around a query are at
// least (R*2^k - 1) fine units away: the bound below which a near-phase
// winner is final.
__device__ void set_far(CutGeom& C, double f) {
  const double gap = ldexp((double)C.R, C.k) - 1.0;
  const double lb2 = gap > 0.0 ? gap * gap * f * f : 0.0;
  C.far64 = lb2 * (1.0 - 1e-9);
  const double l32 = lb2 * (1.0 - 1e-5) - 0x1p-100;
  C.far32 = l32 <= 0.0 ? 0.0f : (l32 >= 3.0e38 ? 3.0e38f : __double2float_rd(l32));
}

__device__ void choose_level(CutGeom& C, const GridGeom* geom, int rpref) {
  const double f = geom->f;
  const int B = geom->B;
  const double Dd = floor(C.dc * geom->inv_f * (1.0 + 1e-9) + 1e-6) + 1.0;
  const int g = geom->g;
  const int rmax = g >= 4 ? 1 : (g == 3 ? 2 : (g == 2 ? 5 : 16));  // (2R+1)^g <= kMaxUnion cells
  int k = B, R = 1;
  double best = INFINITY;
  for (int r = 1; r <= rmax; ++r) {
    if (rpref > 0 && r > rpref) break;
    if (rpref == 0 && r > (g >= 3 ? 2 : 3)) break;
    int kk = 0;
    while (kk < B && ldexp((double)r, kk) < Dd) ++kk;
    const int rr = (int)fmax(1.0, ceil(Dd / ldexp(1.0, kk)));
    if (rr > rmax) continue;
    const double side = (2.0 * rr + 1.0) * ldexp(1.0, kk);
    const bool take = rpref > 0 ? (kk < k || !(best < INFINITY))
                                : side < (best < INFINITY ? 0.8 * best : INFINITY);
    if (take) {
      best = side;
      k = kk;
      R = rr;
    }
  }
  if (!(best < INFINITY)) {  // the cutoff exceeds the whole box: one cell
    k = B;
    R = 1;
  }
  C.k = k;
  C.R = R;
  // density prune: squared lower bound in fine units vs d_cut^2 / f^2
  double pf = C.dc2 * (1.0 + 1e-6) / (f * f) * (1.0 + 1e-6);
  C.prune_fine = pf >= 3.0e38 ? INFINITY : __double2float_ru(pf);
  set_far(C, f);
}

// The near-dependent search on cells `shift` levels finer than the density's,
// with the same block radius: a block 2^shift times narrower, so fewer
// candidates per query and more queries left to the tree search.
__global__ void k_near_level(ClassView cv, CutGeom* cuts, int shift) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.ninst) return;
  CutGeom& C = cuts[i];
  C.k = C.k > shift ? C.k - shift : 0;
  set_far(C, cv.geom[i].f);
}

// Per (instance, cutoff) search parameters, one thread each.  cuts is
// [ncut][ninst].
__global__ void k_setup_cuts(ClassView cv, CutGeom* cuts, int ncut, const CutHost* __restrict__ hc,
                             CutArgs args) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cv.ninst * (uint32_t)ncut) return;
  const uint32_t i = t / ncut;
  const int c = (int)(t - i * ncut);
  const CutHost H = hc ? hc[(size_t)i * ncut + c] : args.h[c];
  CutGeom& C = cuts[(size_t)c * cv.ninst + i];
  C.dc = H.dc;
  C.dc2 = H.dc2;
  C.t_in = H.t_in;
  C.t_out = H.t_out;
  C.band_mul = H.band_mul;
  C.band_add = H.band_add;
  C.skip = H.skip;
  choose_level(C, cv.geom + i, 0);
}

// The level and radius of one cutoff of every instance again, with a
// preferred block radius.
__global__ void k_set_radius(ClassView cv, CutGeom* cuts, int rpref) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cv.ninst) return;
  choose_level(cuts[i], cv.geom + i, rpref);
}

// Sort key of every point: (instance << S) | fine-grid Morton code; the
// payload is the point's class position.
template <typename T, int G>
__global__ void k_codes(const T* __restrict__ pts, ClassView cv,
                        unsigned long long* __restrict__ codes, uint32_t* __restrict__ ids) {
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint64_t total = (uint64_t)cv.nchunk * 32u;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i, p0, end;
    cv.chunk((uint32_t)(e >> 5), i, p0, end);
    const uint32_t p = p0 + (uint32_t)(e & 31u);
    if (p >= end) continue;
    const InstDev I = cv.instance(i);
    const GridGeom* geom = cv.geom + i;
    const double inv_f = geom->inv_f;
    const uint32_t cmax = (1u << geom->B) - 1u;
    const T* row = pts + I.coord + (size_t)(p - I.start) * I.d;
    uint32_t c[G];
#pragma unroll
    for (int a = 0; a < G; ++a) {
      const double x = (double)(float)row[a];
      const double v = (x - geom->org[a]) * inv_f;
      // float-to-integer conversion clamps to [0, 2^32 - 1] (NaN to 0), so
      // only the upper clamp is left, in integer arithmetic (binary64 is
      // the slow pipe on this chip)
      const uint32_t ci = __double2uint_rz(v);
      c[a] = ci < cmax ? ci : cmax;
    }
    codes[p] = (ib ? ((unsigned long long)i << S) : 0ull) | morton<G>(c);
    ids[p] = p;
  }
}

// Points into key order, converted to float and zero padded to DP; sid gets
// each sorted point's output index.
template <typename T, int DP>
__global__ void k_gather(const T* __restrict__ pts, ClassView cv,
                         const unsigned long long* codes_a, const unsigned long long* codes_b,
                         const uint32_t* ids_a, const uint32_t* ids_b,
                         float* __restrict__ spts, unsigned long long* __restrict__ scode,
                         uint32_t* __restrict__ sid) {
  const int S = cv.cls->S, ib = cv.cls->ib;
  const bool odd = sort_passes(S, ib) & 1;
  const unsigned long long* __restrict__ ck = odd ? codes_b : codes_a;
  const uint32_t* __restrict__ ci = odd ? ids_b : ids_a;
  const uint32_t n = cv.N;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned long long key = ck[p];
    uint32_t inst = key_inst(key, S, ib);
    uint32_t o = ci[p];
    if (inst >= cv.ninst) {
      set_status(cv.cls->status, kStatusIndex);
      inst = 0;
    }
    const InstDev I = cv.instance(inst);
    if (o < I.start || o >= I.start + I.n) {
      set_status(cv.cls->status, kStatusIndex);
      o = I.start;
    }
    const uint32_t local = o - I.start;
    const T* row = pts + I.coord + (size_t)local * I.d;
    float x[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = (k < I.d) ? (float)row[k] : 0.f;
    if constexpr (DP == 2) {
      reinterpret_cast<float2*>(spts)[p] = make_float2(x[0], x[1]);
    } else if constexpr (DP == 4) {
      reinterpret_cast<float4*>(spts)[p] = make_float4(x[0], x[1], x[2], x[3]);
    } else {
      float4* q = reinterpret_cast<float4*>(spts) + 2 * (size_t)p;
      q[0] = make_float4(x[0], x[1], x[2], x[3]);
      q[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
    scode[p] = key;
    sid[p] = (uint32_t)(I.out + local);
  }
}

// ---- occupied cells of level k ------------------------------------------------

// Hash key of the level-k cell holding sorted key `key` of instance `inst`.
__device__ __forceinline__ unsigned long long key_cell(unsigned long long key, int S, int ib,
                                                      int shift) {
  return ib ? (((key >> S) << S) | (key_code(key, S, ib) >> shift)) : (key >> shift);
}

__device__ __forceinline__ int cell_shift(const ClassView& cv, const CutGeom* __restrict__ cuts,
                                          unsigned long long key, int S, int ib, int g) {
  uint32_t i = key_inst(key, S, ib);
  if (i >= cv.ninst) i = 0;
  return g * cuts[i].k;
}

__global__ void k_cells_count(const unsigned long long* __restrict__ scode, ClassView cv, int g,
                              const CutGeom* __restrict__ cuts, HashInfo* hi) {
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t n = cv.N;
  uint32_t local = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned long long key = scode[p];
    const int sh = cell_shift(cv, cuts, key, S, ib, g);
    const unsigned long long c = key_cell(key, S, ib, sh);
    local += (p == 0 || key_cell(scode[p - 1], S, ib, sh) != c) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(&hi->m, local);
}

__global__ void k_hash_size(HashInfo* hi, uint32_t hcap) {
  uint32_t want = 2u * hi->m;
  uint32_t t = 16;
  while (t < want && t < hcap) t <<= 1;
  hi->hmask = t - 1;
}

__global__ void k_hash_clear(unsigned long long* __restrict__ hkeys, const HashInfo* __restrict__ hi) {
  const uint32_t T = hi->hmask + 1;
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < T; h += gridDim.x * blockDim.x)
    hkeys[h] = kEmpty;
}

// The first point of a cell records its start, the last its end; both find
// the same slot by probing with compare-and-swap on the key.
__global__ void k_hash_insert(const unsigned long long* __restrict__ scode, ClassView cv, int g,
                              const CutGeom* __restrict__ cuts, const HashInfo* __restrict__ hi,
                              unsigned long long* hkeys, uint2* hvals) {
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t n = cv.N;
  const uint32_t mask = hi->hmask;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const unsigned long long key = scode[p];
    const int sh = cell_shift(cv, cuts, key, S, ib, g);
    const unsigned long long c = key_cell(key, S, ib, sh);
    const bool first = (p == 0) || (key_cell(scode[p - 1], S, ib, sh) != c);
    const bool last = (p == n - 1) || (key_cell(scode[p + 1], S, ib, sh) != c);
    if (!first && !last) continue;
    uint32_t h = hash_slot(c, mask);
    bool placed = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      unsigned long long prev = atomicCAS(&hkeys[h], kEmpty, c);
      if (prev == kEmpty || prev == c) {
        if (first) hvals[h].x = p;
        if (last) hvals[h].y = p + 1;
        placed = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!placed) set_status(cv.cls->status, kStatusHashFull);
  }
}

// Chunk tables of a multi-instance class: block b writes the chunks of
// instance b (grid-stride over instances).
__global__ void k_chunks(const InstDev* __restrict__ inst, uint32_t ninst, uint32_t* chunk_inst,
                         uint32_t* chunk_pos) {
  for (uint32_t i = blockIdx.x; i < ninst; i += gridDim.x) {
    const InstDev I = inst[i];
    const uint32_t nc = (I.n + 31) / 32;
    for (uint32_t j = threadIdx.x; j < nc; j += blockDim.x) {
      chunk_inst[I.chunk0 + j] = i;
      chunk_pos[I.chunk0 + j] = I.start + 32 * j;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side constants of a cutoff: the float32 filter thresholds and the
// ambiguity band, derived from the standard rounding-error bound of a sum of
// DP squared differences, |s32 - s| <= gamma_{DP+2} s + eta, and of the
// canonical binary64 value, |s64 - s| <= gamma64_{DP+2} s.

static float round_down_f(double x) {
  if (x >= 3.0e38) return 3.0e38f;
  if (x <= -3.0e38) return -3.0e38f;
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
}
static float round_up_f(double x) {
  if (x >= 3.0e38) return INFINITY;
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

CutHost make_cut_host(double d_cut, int dp) {
  CutHost h;
  h.dc = d_cut;
  h.dc2 = d_cut * d_cut;
  const double m = dp + 2;
  const double u32 = 0x1p-24, u64 = 0x1p-53;
  const double g32 = m * u32 / (1.0 - m * u32);
  const double g64 = m * u64 / (1.0 - m * u64);
  const double eta = 0x1p-120;
  const double safety = 1e-12;
  h.t_in = round_down_f(h.dc2 * (1.0 - g32) / (1.0 + g64) * (1.0 - safety) - eta);
  h.t_out = round_up_f(h.dc2 * (1.0 + g32) / (1.0 - g64) * (1.0 + safety) + eta);
  double rho_band = (1.0 + g32) * (1.0 + g64) / ((1.0 - g32) * (1.0 - g64)) * (1.0 + safety);
  h.band_mul = round_up_f(rho_band);
  h.band_add = round_up_f(eta * (rho_band + 1.0) * (1.0 + safety));
  h.skip = 0;
  h.pad = 0;
  return h;
}

void launch_class_init(const ClassView& cv, int g, int ib, int bcap, int* status, cudaStream_t st) {
  k_class_init<<<grid_for(cv.ninst), kThreads, 0, st>>>(cv, g, ib, bcap, status);
  count_launches(1);
}

void launch_chunks(const ClassView& cv, uint32_t* chunk_inst, uint32_t* chunk_pos, cudaStream_t st) {
  if (!cv.inst || cv.ninst == 0) return;
  k_chunks<<<grid_for(cv.ninst, 1, sm_count() * 16u), 128, 0, st>>>(cv.inst, cv.ninst, chunk_inst, chunk_pos);
  count_launches(1);
}

void launch_near_level(const ClassView& cv, CutGeom* cuts, int shift, cudaStream_t st) {
  if (shift <= 0) return;
  k_near_level<<<grid_for(cv.ninst), kThreads, 0, st>>>(cv, cuts, shift);
  count_launches(1);
}

void launch_set_radius(const ClassView& cv, CutGeom* cuts, int rpref, cudaStream_t st) {
  k_set_radius<<<grid_for(cv.ninst), kThreads, 0, st>>>(cv, cuts, rpref);
  count_launches(1);
}

void launch_bbox(const void* pts, int dtype, const ClassView& cv, int g, cudaStream_t st) {
  if (cv.N == 0) return;
  const unsigned grid = grid_for((uint64_t)cv.nchunk * 32u, kThreads, sm_count() * 4u);
  if (dtype == 0)
    k_bbox<int32_t><<<grid, kThreads, 0, st>>>((const int32_t*)pts, cv, g);
  else
    k_bbox<float><<<grid, kThreads, 0, st>>>((const float*)pts, cv, g);
  count_launches(1);
}

void launch_setup(const ClassView& cv, CutGeom* cuts, int ncut, const CutHost* hc_dev,
                  const CutHost* hc_host, cudaStream_t st) {
  CutArgs a;
  if (!hc_dev)
    for (int c = 0; c < ncut && c < kCutChunk; ++c) a.h[c] = hc_host[c];
  k_setup_geom<<<grid_for(cv.ninst), kThreads, 0, st>>>(cv, ncut, hc_dev, a);
  k_setup_cuts<<<grid_for((uint64_t)cv.ninst * ncut), kThreads, 0, st>>>(cv, cuts, ncut, hc_dev, a);
  count_launches(2);
}

template <typename T>
static void codes_t(const T* pts, const ClassView& cv, int g, unsigned long long* codes,
                    uint32_t* ids, cudaStream_t st) {
  const unsigned grid = grid_for((uint64_t)cv.nchunk * 32u);
  if (g == 1) k_codes<T, 1><<<grid, kThreads, 0, st>>>(pts, cv, codes, ids);
  else if (g == 2) k_codes<T, 2><<<grid, kThreads, 0, st>>>(pts, cv, codes, ids);
  else if (g == 3) k_codes<T, 3><<<grid, kThreads, 0, st>>>(pts, cv, codes, ids);
  else k_codes<T, 4><<<grid, kThreads, 0, st>>>(pts, cv, codes, ids);
  count_launches(1);
}

void launch_codes(const void* pts, int dtype, const ClassView& cv, int g, unsigned long long* codes,
                  uint32_t* ids, cudaStream_t st) {
  if (cv.N == 0) return;
  if (dtype == 0) codes_t((const int32_t*)pts, cv, g, codes, ids, st);
  else codes_t((const float*)pts, cv, g, codes, ids, st);
}

template <typename T>
static void gather_t(const T* pts, const ClassView& cv, int dp, const unsigned long long* ca,
                     const unsigned long long* cb, const uint32_t* ia, const uint32_t* ib,
                     float* spts, unsigned long long* scode, uint32_t* sid, cudaStream_t st) {
  const unsigned grid = grid_for(cv.N);
  if (dp == 2) k_gather<T, 2><<<grid, kThreads, 0, st>>>(pts, cv, ca, cb, ia, ib, spts, scode, sid);
  else if (dp == 4) k_gather<T, 4><<<grid, kThreads, 0, st>>>(pts, cv, ca, cb, ia, ib, spts, scode, sid);
  else k_gather<T, 8><<<grid, kThreads, 0, st>>>(pts, cv, ca, cb, ia, ib, spts, scode, sid);
  count_launches(1);
}

void launch_gather(const void* pts, int dtype, const ClassView& cv, int dp,
                   const unsigned long long* codes_a, const unsigned long long* codes_b,
                   const uint32_t* ids_a, const uint32_t* ids_b, float* spts,
                   unsigned long long* scode, uint32_t* sid, cudaStream_t st) {
  if (cv.N == 0) return;
  if (dtype == 0)
    gather_t((const int32_t*)pts, cv, dp, codes_a, codes_b, ids_a, ids_b, spts, scode, sid, st);
  else
    gather_t((const float*)pts, cv, dp, codes_a, codes_b, ids_a, ids_b, spts, scode, sid, st);
}

void launch_cells(const unsigned long long* scode, const ClassView& cv, int g, const CutGeom* cuts,
                  HashInfo* hi, unsigned long long* hkeys, uint2* hvals, uint32_t hcap,
                  cudaStream_t st) {
  if (cv.N == 0) return;
  const unsigned grid = grid_for(cv.N);
  cudaMemsetAsync(hi, 0, sizeof(HashInfo), st);
  k_cells_count<<<grid, kThreads, 0, st>>>(scode, cv, g, cuts, hi);
  k_hash_size<<<1, 1, 0, st>>>(hi, hcap);
  k_hash_clear<<<grid_for(hcap), kThreads, 0, st>>>(hkeys, hi);
  k_hash_insert<<<grid, kThreads, 0, st>>>(scode, cv, g, cuts, hi, hkeys, hvals);
  count_launches(4);
}

}  // namespace dpc
