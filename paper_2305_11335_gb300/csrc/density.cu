// density.cu -- rho_i = |{j : D(x_i, x_j) <= d_cut}| (Definition 1).
//
// One thread per point, points taken in Morton order so a warp covers a
// compact patch of space and its neighbour cells are shared in L1.  Each
// thread visits the (2R+1)^g level-k cells around its own (R = 1 when the
// cell side is at least d_cut), skips cells whose conservative lower bound
// already exceeds d_cut (the subtree pruning idea of Section 6.1 applied to
// grid cells), and counts the points of the others:
//   FP32_CERT: s32 <= t_in counts, s32 > t_out does not, anything between is
//              re-evaluated with the canonical binary64 distance (rare: the
//              band is about 1e-6 of d_cut^2 wide);
//   FP64:      every pair is evaluated in binary64.
// Both give exactly the binary64 count.  The kernel also writes the order key
// of every sorted point, (rho << 32) | ~id.
#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 256;

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads)
k_density(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
          const uint32_t* __restrict__ sid, uint32_t n, const GridGeom* __restrict__ geom,
          const CutGeom* __restrict__ cut, const unsigned long long* __restrict__ hkeys,
          const uint2* __restrict__ hvals, int32_t* __restrict__ rho_out,
          unsigned long long* __restrict__ skey, Counters* ctr) {
  const int k = cut->k;
  const int R = cut->R;
  const int W = 2 * R + 1;
  const int shift = G * k;
  const int cmax = (1 << (geom->B - k)) - 1;
  const float cell_fine = (float)(1u << k);
  const double dc2 = cut->dc2;
  const float t_in = cut->t_in, t_out = cut->t_out;
  const float prune = cut->prune_fine;
  const uint32_t hmask = cut->hmask;
  const double inv_f = geom->inv_f;
  double org[G];
#pragma unroll
  for (int a = 0; a < G; ++a) org[a] = geom->org[a];
  int ncell = 1;
  for (int a = 0; a < G; ++a) ncell *= W;

  unsigned long long band = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const Pt<DP> q = load_pt<DP>(spts, p);
    float u[G];
#pragma unroll
    for (int a = 0; a < G; ++a) u[a] = (float)(((double)q.x[a] - org[a]) * inv_f);
    uint32_t c0[G];
    unmorton<G>(scode[p] >> shift, c0);
    int32_t count = 0;
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
        const float hi = lo + cell_fine - 1.f;
        const float l = fmaxf(fmaxf(lo - 1.f - u[a], u[a] - hi - 2.f), 0.f);
        lb2 = fmaf(l, l, lb2);
      }
      if (!inside || lb2 > prune) continue;
      const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, morton<G>(c)), n);
      for (uint32_t t = run.x; t < run.y; ++t) {
        const Pt<DP> x = load_pt<DP>(spts, t);
        if constexpr (F64) {
          count += dist64<DP>(q, x) <= dc2;
        } else {
          const float s = dist32<DP>(q, x);
          if (s <= t_in) {
            ++count;
          } else if (s <= t_out) {
            ++band;
            count += dist64<DP>(q, x) <= dc2;
          }
        }
      }
    }
    const uint32_t id = sid[p];
    rho_out[id] = count;
    skey[p] = order_key(count, id);
  }
  if constexpr (!F64) {
    for (int o = 16; o > 0; o >>= 1) band += __shfl_xor_sync(0xffffffffu, band, o);
    if ((threadIdx.x & 31) == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

__global__ void k_keys_from_rho(const int32_t* __restrict__ rho, const uint32_t* __restrict__ sid,
                                uint32_t n, unsigned long long* __restrict__ skey) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t id = sid[p];
    skey[p] = order_key(rho[id], id);
  }
}

inline unsigned grid_for(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152u * 64u) b = 152u * 64u;
  return (unsigned)b;
}

template <int DP, int G>
void density_dg(bool fp64, const float* spts, const unsigned long long* scode, const uint32_t* sid,
                uint32_t n, const GridGeom* geom, const CutGeom* cut,
                const unsigned long long* hkeys, const uint2* hvals, int32_t* rho_out,
                unsigned long long* skey, Counters* ctr, cudaStream_t st) {
  const unsigned grid = grid_for(n);
  if (fp64)
    k_density<DP, G, true><<<grid, kThreads, 0, st>>>(spts, scode, sid, n, geom, cut, hkeys, hvals,
                                                      rho_out, skey, ctr);
  else
    k_density<DP, G, false><<<grid, kThreads, 0, st>>>(spts, scode, sid, n, geom, cut, hkeys, hvals,
                                                       rho_out, skey, ctr);
  count_launches(1);
}

}  // namespace

void launch_density(int dp, int g, bool fp64, const float* spts, const unsigned long long* scode,
                    const uint32_t* sid, uint32_t n, const GridGeom* geom, const CutGeom* cut,
                    const unsigned long long* hkeys, const uint2* hvals, int32_t* rho_out,
                    unsigned long long* skey, Counters* ctr, cudaStream_t st) {
  if (n == 0) return;
  if (g == 1) density_dg<2, 1>(fp64, spts, scode, sid, n, geom, cut, hkeys, hvals, rho_out, skey, ctr, st);
  else if (g == 2) density_dg<2, 2>(fp64, spts, scode, sid, n, geom, cut, hkeys, hvals, rho_out, skey, ctr, st);
  else if (dp == 4) density_dg<4, 3>(fp64, spts, scode, sid, n, geom, cut, hkeys, hvals, rho_out, skey, ctr, st);
  else density_dg<8, 3>(fp64, spts, scode, sid, n, geom, cut, hkeys, hvals, rho_out, skey, ctr, st);
}

void launch_keys_from_rho(const int32_t* rho, const uint32_t* sid, uint32_t n,
                          unsigned long long* skey, cudaStream_t st) {
  if (n == 0) return;
  k_keys_from_rho<<<grid_for(n), kThreads, 0, st>>>(rho, sid, n, skey);
  count_launches(1);
}

}  // namespace dpc
