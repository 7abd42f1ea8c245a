// density.cu -- rho_i = |{j : D(x_i, x_j) <= d_cut}| (Definition 1).
//
// A warp owns 32 consecutive Morton-sorted points.  For each level-k cell
// they fall into (a "segment"), the warp looks up the (2R+1)^g cells of the
// cell's block in parallel and stages their points in shared memory (in
// windows of kCap).  A segment of 32 queries (one dense cell) runs one query
// per lane over the window with broadcast reads; smaller segments run 4
// queries at a time with 8 lanes each.
//   FP32_CERT: s32 <= t_in counts, s32 > t_out does not.  Pairs in between
//              (about 1e-6 of d_cut^2 wide) are counted with the canonical
//              binary64 distance in a separate pass that runs only when a
//              warp meets one, so the hot loop stays float32.
//   FP64:      every pair is evaluated in binary64.
// Both give exactly the binary64 count.  The kernel also writes the order key
// of every sorted point, (rho << 32) | ~id.
#include "block.cuh"
#include "internal.h"

namespace dpc {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

template <int DP>
constexpr int density_cap() { return DP == 8 ? 256 : 512; }

// Exact count of the band pairs among window candidates t0, t0+step, ... < T.
template <int DP>
__device__ __noinline__ int2 band_count(const float* __restrict__ wpts, uint32_t t0, uint32_t T,
                                        uint32_t step, Pt<DP> q, float t_in, float t_out,
                                        double dc2) {
  int in = 0, seen = 0;
  for (uint32_t t = t0; t < T; t += step) {
    const Pt<DP> x = window_pt<DP>(wpts, t);
    const float s32 = dist32<DP>(q, x);
    if (s32 > t_in && s32 <= t_out) {
      ++seen;
      in += dist64<DP>(q, x) <= dc2;
    }
  }
  return make_int2(in, seen);
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads)
k_density(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
          const uint32_t* __restrict__ sid, uint32_t n, const GridGeom* __restrict__ geom,
          const CutGeom* __restrict__ cut, const unsigned long long* __restrict__ hkeys,
          const uint2* __restrict__ hvals, int32_t* __restrict__ rho_out,
          unsigned long long* __restrict__ skey, Counters* ctr) {
  constexpr int kCap = density_cap<DP>();
  __shared__ __align__(16) float smem[kWarps * kCap * DP];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* wpts = smem + wib * kCap * DP;

  const int k = cut->k;
  const int R = cut->R;
  const int shift = G * k;
  const int cmax = (1 << (geom->B - k)) - 1;
  const double dc2 = cut->dc2;
  const float t_in = cut->t_in, t_out = cut->t_out;
  const uint32_t hmask = cut->hmask;
  const int sub = lane & 7;     // lane within its query group
  const int grp = lane >> 3;    // query group 0..3

  unsigned long long band = 0;
  const uint32_t nchunk = (n + 31) / 32;
  for (uint32_t ch = blockIdx.x * kWarps + wib; ch < nchunk; ch += gridDim.x * kWarps) {
    const uint32_t p0 = ch * 32;
    const uint32_t p = p0 + lane;
    const bool valid = p < n;
    Pt<DP> me;
#pragma unroll
    for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
    if (valid) me = load_pt<DP>(spts, p);
    const unsigned long long mycell = valid ? (scode[p] >> shift) : ~0ull;
    const int nvalid = (int)min(32u, n - p0);
    int32_t count = 0;
    int s = 0;
    while (s < nvalid) {
      const unsigned long long cell = __shfl_sync(kFull, mycell, s);
      const int e = s + __popc(__ballot_sync(kFull, mycell == cell));
      uint32_t c0[G];
      unmorton<G>(cell, c0);
      BlockRuns br;
      lookup_block<G>(c0, R, cmax, hkeys, hvals, hmask, n, lane, br);
      for (uint32_t w0 = 0; w0 < br.total; w0 += kCap) {
        const uint32_t T = min((uint32_t)kCap, br.total - w0);
        __syncwarp();
        stage_window<DP, false>(br, w0, kCap, spts, nullptr, wpts, nullptr, lane);
        __syncwarp();
        if (e - s == 32) {
          // one query per lane, every lane reads the same candidate; c counts
          // s32 <= t_in (certainly within d_cut), c2 counts s32 <= t_out
          int32_t c = 0, c2 = 0;
#pragma unroll 4
          for (uint32_t t = 0; t < T; ++t) {
            const Pt<DP> x = window_pt<DP>(wpts, t);
            if constexpr (F64) {
              c += dist64<DP>(me, x) <= dc2;
            } else {
              const float s32 = dist32<DP>(me, x);
              c += s32 <= t_in;
              c2 += s32 <= t_out;
            }
          }
          if constexpr (!F64) {
            if (__any_sync(kFull, c2 != c)) {
              const int2 r = band_count<DP>(wpts, 0, T, 1, me, t_in, t_out, dc2);
              c += r.x;
              band += r.y;
            }
          }
          count += c;
          continue;
        }
        for (int qb = s; qb < e; qb += 4) {
          const int qi = qb + grp;
          const Pt<DP> q = shfl_pt<DP>(me, qi < e ? qi : s);
          int32_t c = 0, c2 = 0;
#pragma unroll 2
          for (uint32_t t = sub; t < T; t += 8) {
            const Pt<DP> x = window_pt<DP>(wpts, t);
            if constexpr (F64) {
              c += dist64<DP>(q, x) <= dc2;
            } else {
              const float s32 = dist32<DP>(q, x);
              c += s32 <= t_in;
              c2 += s32 <= t_out;
            }
          }
          if constexpr (!F64) {
            if (__any_sync(kFull, c2 != c)) {
              const int2 r = band_count<DP>(wpts, sub, T, 8, q, t_in, t_out, dc2);
              c += r.x;
              if (qi < e) band += r.y;
            }
          }
          c += __shfl_xor_sync(kFull, c, 4);
          c += __shfl_xor_sync(kFull, c, 2);
          c += __shfl_xor_sync(kFull, c, 1);
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int v = __shfl_sync(kFull, c, g * 8);
            if (lane == qb + g && qb + g < e) count += v;
          }
        }
      }
      s = e;
    }
    if (valid) {
      const uint32_t id = sid[p];
      rho_out[id] = count;
      skey[p] = order_key(count, id);
    }
  }
  if constexpr (!F64) {
    for (int o = 16; o > 0; o >>= 1) band += __shfl_xor_sync(kFull, band, o);
    if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

__global__ void k_keys_from_rho(const int32_t* __restrict__ rho, const uint32_t* __restrict__ sid,
                                uint32_t n, unsigned long long* __restrict__ skey) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t id = sid[p];
    skey[p] = order_key(rho[id], id);
  }
}

inline unsigned grid_for(uint64_t items, int per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, int G>
void density_dg(bool fp64, const float* spts, const unsigned long long* scode, const uint32_t* sid,
                uint32_t n, const GridGeom* geom, const CutGeom* cut,
                const unsigned long long* hkeys, const uint2* hvals, int32_t* rho_out,
                unsigned long long* skey, Counters* ctr, cudaStream_t st) {
  const unsigned grid = grid_for((n + 31) / 32, kWarps, 152u * 64u);
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
  k_keys_from_rho<<<grid_for(n, 256, 152u * 16u), 256, 0, st>>>(rho, sid, n, skey);
  count_launches(1);
}

}  // namespace dpc
