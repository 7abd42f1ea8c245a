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

inline unsigned grid_for(uint64_t n, int threads = kThreads, unsigned cap = 152u * 16u) {
  uint64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

__global__ void k_geom_init(GridGeom* geom, int* status, int g) {
  geom->g = g;
  geom->status = status;
  for (int a = 0; a < 3; ++a) {
    geom->bbox_ord[a] = 0xffffffffu;  // min accumulators
    geom->bbox_ord[3 + a] = 0u;       // max accumulators
  }
}

// Bounding box of the gridded axes and the coordinate range check.
template <typename T>
__global__ void k_bbox(const T* __restrict__ pts, uint32_t n, int d, int g, GridGeom* geom) {
  float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
  float mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  int bad = 0;
  const uint64_t total = (uint64_t)n * d;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    T v = pts[e];
    float x;
    if constexpr (std::is_integral<T>::value) {
      bad |= (v > (1 << 24)) | (v < -(1 << 24));
      x = (float)v;
    } else {
      x = (float)v;
      bad |= !(fabsf(x) <= 1.152921504606846976e18f);  // 2^60; false for NaN
    }
    int a = (int)(e % (uint64_t)d);
    if (a < g) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k == a) { mn[k] = fminf(mn[k], x); mx[k] = fmaxf(mx[k], x); }
    }
  }
  // warp reduce, block reduce through shared memory, one atomic per block
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    }
  }
  __shared__ float s_mn[32][3], s_mx[32][3];
  __shared__ int s_bad;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { s_mn[w][k] = mn[k]; s_mx[w][k] = mx[k]; }
  }
  if (bad) s_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < g; ++k) {
      float a = s_mn[0][k], b = s_mx[0][k];
      for (int j = 1; j < nw; ++j) { a = fminf(a, s_mn[j][k]); b = fmaxf(b, s_mx[j][k]); }
      if (a <= b) {
        atomicMin(&geom->bbox_ord[k], float_ord(a));
        atomicMax(&geom->bbox_ord[3 + k], float_ord(b));
      }
    }
    if (s_bad) set_status(geom->status, kStatusBadCoord);
  }
}

// Grid geometry from the bounding box.
//
// Fine grid: the fine cell is 1/8 of the smallest cutoff (times 1 + 2^-20),
// so the level-3 cell is just wider than d_cut and the 3^g block around it
// holds every point within d_cut with the least volume a cell grid allows.
// At most kMaxBits bits per axis keep fine-unit coordinates exact to 1/8 cell
// in float32; a wider bounding box gets a coarser fine cell instead.
// A point's fine index c = floor((x - org) * inv_f) is within 1e-9 cells of the
// exact real value, so its real position lies in [c - 0.5, c + 1.5) fine units;
// every bound below is derived from that interval.
__global__ void k_setup_geom(GridGeom* geom, double dcmin) {
  if (threadIdx.x != 0) return;
  const int g = geom->g;
  double E = 0.0;
  for (int a = 0; a < g; ++a) {
    uint32_t lo = geom->bbox_ord[a], hi = geom->bbox_ord[3 + a];
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
    if (f_fit > 0.0 && E / f_fit < ldexp(1.0, kMaxBits) * (1.0 - 0x1p-20)) {
      f = f_fit;
      B = 1;
      while (ldexp(f, B) <= E * (1.0 + 0x1p-30)) ++B;  // E / f < 2^B with margin
    } else {
      B = kMaxBits;
      f = ldexp(E, -B) * (1.0 + 0x1p-20);
    }
  }
  geom->B = B;
  geom->f = f;
  geom->inv_f = 1.0 / f;
  geom->f2 = __double2float_rd(f * f);
  geom->nbits = g * B;
  geom->npass = (g * B + 7) / 8;
}

// Per-cutoff search parameters: the grid level k whose cells are at least
// d_cut wide (so the (2R+1)^g block with R = 1 holds every point within
// d_cut), the density prune bound and the far bound of the dependent search.
constexpr int kCutChunk = 16;
struct CutArgs {
  CutHost h[kCutChunk];
};
__global__ void k_setup_cuts(const GridGeom* __restrict__ geom, CutGeom* cuts, int ncut, CutArgs a) {
  const int c = threadIdx.x;
  if (c >= ncut) return;
  const double f = geom->f;
  const int B = geom->B;
  CutGeom& C = cuts[c];
  C.dc = a.h[c].dc;
  C.dc2 = a.h[c].dc2;
  C.t_in = a.h[c].t_in;
  C.t_out = a.h[c].t_out;
  C.band_mul = a.h[c].band_mul;
  C.band_add = a.h[c].band_add;
  // Two points within d_cut differ by at most D fine indices on each axis.
  // Choose the level k and block radius R (R * 2^k >= D).  R = 1 (the 3^g
  // block of cells at least d_cut wide) unless a larger R on finer cells
  // shrinks the block side by more than 20%, which pays for its extra cell
  // lookups (it happens when d_cut falls just above a power-of-two multiple
  // of the fine cell, e.g. the larger cutoffs of a sweep).
  const double Dd = floor(C.dc * geom->inv_f * (1.0 + 1e-9) + 1e-6) + 1.0;
  const int g = geom->g;
  const int rmax = g == 3 ? 2 : 3;  // (2R+1)^g <= 125 cells
  int k = B, R = 1;
  double best = INFINITY;
  for (int r = 1; r <= rmax; ++r) {
    int kk = 0;
    while (kk < B && ldexp((double)r, kk) < Dd) ++kk;
    const int rr = (int)fmax(1.0, ceil(Dd / ldexp(1.0, kk)));
    if (rr > rmax) continue;
    const double side = (2.0 * rr + 1.0) * ldexp(1.0, kk);
    if (side < (best < INFINITY ? 0.8 * best : INFINITY)) {
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
  // points outside the (2R+1)^g block are at least (R*2^k - 1) fine units away
  double gap = ldexp((double)R, k) - 1.0;
  double lb2 = gap > 0.0 ? gap * gap * f * f : 0.0;
  C.far64 = lb2 * (1.0 - 1e-9);
  double l32 = lb2 * (1.0 - 1e-5) - 0x1p-100;
  C.far32 = l32 <= 0.0 ? 0.0f : (l32 >= 3.0e38 ? 3.0e38f : __double2float_rd(l32));
  C.m = 0;
  C.hmask = 0;
}

// Fine-grid Morton code of every point.
template <typename T, int G>
__global__ void k_codes(const T* __restrict__ pts, uint32_t n, int d, const GridGeom* __restrict__ geom,
                        unsigned long long* __restrict__ codes, uint32_t* __restrict__ ids) {
  const double inv_f = geom->inv_f;
  const uint32_t cmax = (1u << geom->B) - 1u;
  double org[G];
#pragma unroll
  for (int a = 0; a < G; ++a) org[a] = geom->org[a];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t c[G];
#pragma unroll
    for (int a = 0; a < G; ++a) {
      double x = (double)(float)pts[(size_t)i * d + a];
      double v = (x - org[a]) * inv_f;
      v = fmin(fmax(v, 0.0), (double)cmax);
      c[a] = (uint32_t)v;
    }
    codes[i] = morton<G>(c);
    ids[i] = i;
  }
}

// Points into Morton order, converted to float and zero padded to DP.
template <typename T, int DP>
__global__ void k_gather(const T* __restrict__ pts, uint32_t n, int d, const GridGeom* __restrict__ geom,
                         const unsigned long long* codes_a, const unsigned long long* codes_b,
                         const uint32_t* ids_a, const uint32_t* ids_b,
                         float* __restrict__ spts, unsigned long long* __restrict__ scode,
                         uint32_t* __restrict__ sid) {
  const bool odd = geom->npass & 1;
  const unsigned long long* __restrict__ ck = odd ? codes_b : codes_a;
  const uint32_t* __restrict__ ci = odd ? ids_b : ids_a;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    uint32_t o = ci[p];
    if (o >= n) {
      set_status(geom->status, kStatusIndex);
      o = 0;
    }
    float x[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = (k < d) ? (float)pts[(size_t)o * d + k] : 0.f;
    if constexpr (DP == 2) {
      reinterpret_cast<float2*>(spts)[p] = make_float2(x[0], x[1]);
    } else if constexpr (DP == 4) {
      reinterpret_cast<float4*>(spts)[p] = make_float4(x[0], x[1], x[2], x[3]);
    } else {
      float4* q = reinterpret_cast<float4*>(spts) + 2 * (size_t)p;
      q[0] = make_float4(x[0], x[1], x[2], x[3]);
      q[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
    scode[p] = ck[p];
    sid[p] = o;
  }
}

// ---- occupied cells of level k ------------------------------------------------

__global__ void k_cells_count(const unsigned long long* __restrict__ scode, uint32_t n,
                              const GridGeom* __restrict__ geom, CutGeom* cut) {
  const int sh = geom->g * cut->k;
  uint32_t local = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    unsigned long long c = scode[p] >> sh;
    local += (p == 0 || (scode[p - 1] >> sh) != c) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(&cut->m, local);
}

__global__ void k_hash_size(CutGeom* cut, uint32_t hcap) {
  uint32_t want = 2u * cut->m;
  uint32_t t = 16;
  while (t < want && t < hcap) t <<= 1;
  cut->hmask = t - 1;
}

__global__ void k_hash_clear(unsigned long long* __restrict__ hkeys, const CutGeom* __restrict__ cut) {
  const uint32_t T = cut->hmask + 1;
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < T; h += gridDim.x * blockDim.x)
    hkeys[h] = kEmpty;
}

// The first point of a cell records its start, the last its end; both find
// the same slot by probing with compare-and-swap on the key.
__global__ void k_hash_insert(const unsigned long long* __restrict__ scode, uint32_t n,
                              const GridGeom* __restrict__ geom, const CutGeom* __restrict__ cut,
                              unsigned long long* hkeys, uint2* hvals) {
  const int sh = geom->g * cut->k;
  const uint32_t mask = cut->hmask;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    unsigned long long c = scode[p] >> sh;
    bool first = (p == 0) || ((scode[p - 1] >> sh) != c);
    bool last = (p == n - 1) || ((scode[p + 1] >> sh) != c);
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
    if (!placed) set_status(geom->status, kStatusHashFull);
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
  return h;
}

void launch_geom_init(GridGeom* geom, int* status, int g, cudaStream_t st) {
  k_geom_init<<<1, 1, 0, st>>>(geom, status, g);
  count_launches(1);
}

void launch_bbox(const void* pts, int dtype, uint32_t n, int d, int g, GridGeom* geom,
                 cudaStream_t st) {
  if (n == 0) return;
  unsigned grid = grid_for((uint64_t)n * d);
  if (dtype == 0)
    k_bbox<int32_t><<<grid, kThreads, 0, st>>>((const int32_t*)pts, n, d, g, geom);
  else
    k_bbox<float><<<grid, kThreads, 0, st>>>((const float*)pts, n, d, g, geom);
  count_launches(1);
}

void launch_setup(GridGeom* geom, CutGeom* cuts, const CutHost* host_cuts, int ncut,
                  cudaStream_t st) {
  double dcmin = INFINITY;
  for (int c = 0; c < ncut; ++c) dcmin = fmin(dcmin, host_cuts[c].dc);
  k_setup_geom<<<1, 32, 0, st>>>(geom, dcmin);
  for (int c0 = 0; c0 < ncut; c0 += kCutChunk) {
    CutArgs a;
    int m = ncut - c0 < kCutChunk ? ncut - c0 : kCutChunk;
    for (int c = 0; c < m; ++c) a.h[c] = host_cuts[c0 + c];
    k_setup_cuts<<<1, 32, 0, st>>>(geom, cuts + c0, m, a);
    count_launches(1);
  }
  count_launches(1);
}

template <typename T>
static void codes_t(const T* pts, uint32_t n, int d, const GridGeom* geom,
                    unsigned long long* codes, uint32_t* ids, cudaStream_t st) {
  unsigned grid = grid_for(n);
  int g = d < 3 ? d : 3;
  if (g == 1) k_codes<T, 1><<<grid, kThreads, 0, st>>>(pts, n, d, geom, codes, ids);
  else if (g == 2) k_codes<T, 2><<<grid, kThreads, 0, st>>>(pts, n, d, geom, codes, ids);
  else k_codes<T, 3><<<grid, kThreads, 0, st>>>(pts, n, d, geom, codes, ids);
  count_launches(1);
}

void launch_codes(const void* pts, int dtype, uint32_t n, int d, const GridGeom* geom,
                  unsigned long long* codes, uint32_t* ids, cudaStream_t st) {
  if (n == 0) return;
  if (dtype == 0) codes_t((const int32_t*)pts, n, d, geom, codes, ids, st);
  else codes_t((const float*)pts, n, d, geom, codes, ids, st);
}

template <typename T>
static void gather_t(const T* pts, uint32_t n, int d, int dp, const GridGeom* geom,
                     const unsigned long long* ca, const unsigned long long* cb, const uint32_t* ia,
                     const uint32_t* ib, float* spts, unsigned long long* scode, uint32_t* sid,
                     cudaStream_t st) {
  unsigned grid = grid_for(n);
  if (dp == 2) k_gather<T, 2><<<grid, kThreads, 0, st>>>(pts, n, d, geom, ca, cb, ia, ib, spts, scode, sid);
  else if (dp == 4) k_gather<T, 4><<<grid, kThreads, 0, st>>>(pts, n, d, geom, ca, cb, ia, ib, spts, scode, sid);
  else k_gather<T, 8><<<grid, kThreads, 0, st>>>(pts, n, d, geom, ca, cb, ia, ib, spts, scode, sid);
  count_launches(1);
}

void launch_gather(const void* pts, int dtype, uint32_t n, int d, int dp, const GridGeom* geom,
                   const unsigned long long* codes_a, const unsigned long long* codes_b,
                   const uint32_t* ids_a, const uint32_t* ids_b, float* spts,
                   unsigned long long* scode, uint32_t* sid, cudaStream_t st) {
  if (n == 0) return;
  if (dtype == 0)
    gather_t((const int32_t*)pts, n, d, dp, geom, codes_a, codes_b, ids_a, ids_b, spts, scode, sid, st);
  else
    gather_t((const float*)pts, n, d, dp, geom, codes_a, codes_b, ids_a, ids_b, spts, scode, sid, st);
}

void launch_cells(const unsigned long long* scode, uint32_t n, const GridGeom* geom, CutGeom* cut,
                  unsigned long long* hkeys, uint2* hvals, uint32_t hcap, cudaStream_t st) {
  if (n == 0) return;
  unsigned grid = grid_for(n);
  k_cells_count<<<grid, kThreads, 0, st>>>(scode, n, geom, cut);
  k_hash_size<<<1, 1, 0, st>>>(cut, hcap);
  k_hash_clear<<<grid_for(hcap), kThreads, 0, st>>>(hkeys, cut);
  k_hash_insert<<<grid, kThreads, 0, st>>>(scode, n, geom, cut, hkeys, hvals);
  count_launches(4);
}

}  // namespace dpc
