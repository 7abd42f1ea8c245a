// block.cuh -- warp-cooperative access to the (2R+1)^g grid block around a
// cell: parallel hash lookups of the neighbour cells and staging of their
// points (and keys) into the warp's shared-memory window.
//
// Work layout shared by the density and near-dependent kernels: a warp owns
// 32 consecutive Morton-sorted points.  They fall into one or more level-k
// cells ("segments", contiguous because the order is by cell); for each
// segment the warp stages the candidates of the cell's block once and runs
// the segment's queries against them, 4 queries at a time with 8 lanes each.
#pragma once

#include "dpc_device.cuh"

namespace dpc {

constexpr int kMaxBlockCells = 128;  // (2R+1)^g <= 125
constexpr int kRunRounds = kMaxBlockCells / 32;
constexpr unsigned kFull = 0xffffffffu;

// Runs of the block's cells: lane l holds the cells with offset index
// l + 32 r.  pre[r] is the run's offset in the concatenated candidate list.
struct BlockRuns {
  uint32_t start[kRunRounds];
  uint32_t len[kRunRounds];
  uint32_t pre[kRunRounds];
  uint32_t total;
  int rounds;  // rounds of 32 cells actually used
};

// floor(x / w) for 0 <= x < 2^10 and w in {1, 3, 5, 7}: x * ceil(2^16 / w) >> 16.
__device__ __forceinline__ int div_small(int x, int inv) { return (x * inv) >> 16; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Look up every cell of the (2R+1)^G block around cell c0 (level-k indices,
// valid range [0, cmax] per axis).
template <int G>
__device__ __forceinline__ void lookup_block(const uint32_t* c0, int R, int cmax,
                                             const unsigned long long* __restrict__ hkeys,
                                             const uint2* __restrict__ hvals, uint32_t hmask,
                                             uint32_t n, int lane, BlockRuns& br) {
  const int W = 2 * R + 1;
  const int invW = (65536 + W - 1) / W;
  int ncell = W;
  if (G >= 2) ncell *= W;
  if (G >= 3) ncell *= W;
  uint32_t total = 0;
  br.rounds = (ncell + 31) >> 5;
#pragma unroll
  for (int r = 0; r < kRunRounds; ++r) {
    br.start[r] = 0;
    br.len[r] = 0;
    br.pre[r] = total;
    if (r >= br.rounds) continue;
    const int o = r * 32 + lane;
    uint32_t st = 0, len = 0;
    if (o < ncell) {
      int rem = o;
      uint32_t c[G];
      bool inside = true;
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const int q = div_small(rem, invW);
        const int ca = (int)c0[a] + (rem - q * W) - R;
        rem = q;
        inside &= (ca >= 0) & (ca <= cmax);
        c[a] = (uint32_t)ca;
      }
      if (inside) {
        const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, morton<G>(c)), n);
        st = run.x;
        len = run.y - run.x;
      }
    }
    const uint32_t incl = warp_incl_scan(len, lane);
    br.start[r] = st;
    br.len[r] = len;
    br.pre[r] = total + incl - len;
    total += __shfl_sync(kFull, incl, 31);
  }
  br.total = total;
}

// Copy candidates [w0, w0 + cap) of the concatenated block list into the
// warp's window: coordinates (DP floats), and for KEYS also order keys.
template <int DP, bool KEYS>
__device__ __forceinline__ void stage_window(const BlockRuns& br, uint32_t w0, uint32_t cap,
                                             const float* __restrict__ spts,
                                             const unsigned long long* __restrict__ skey,
                                             float* __restrict__ wpts,
                                             unsigned long long* __restrict__ wkey, int lane) {
  const uint32_t w1 = w0 + cap;
#pragma unroll
  for (int r = 0; r < kRunRounds; ++r) {
    if (r >= br.rounds) break;
    const uint32_t lo = br.pre[r], hi = br.pre[r] + br.len[r];
    unsigned mask = __ballot_sync(kFull, br.len[r] > 0 && lo < w1 && hi > w0);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t rs = __shfl_sync(kFull, br.start[r], j);
      const uint32_t rlo = __shfl_sync(kFull, lo, j);
      const uint32_t rhi = __shfl_sync(kFull, hi, j);
      const uint32_t a = rlo > w0 ? rlo : w0;
      const uint32_t b = rhi < w1 ? rhi : w1;
      for (uint32_t e = a + lane; e < b; e += 32) {
        const uint32_t src = rs + (e - rlo);
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
  }
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

template <int DP>
__device__ __forceinline__ Pt<DP> shfl_pt(const Pt<DP>& p, int src) {
  Pt<DP> q;
#pragma unroll
  for (int k = 0; k < DP; ++k) q.x[k] = __shfl_sync(kFull, p.x[k], src);
  return q;
}

}  // namespace dpc
