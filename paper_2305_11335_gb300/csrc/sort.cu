// sort.cu -- LSD radix sort of (64-bit code, 32-bit id) pairs by code.
//
// The radix-sort primitive of Section 3.2, used here to put the points in
// Morton order.  One read of the keys counts the digits of every pass
// (k_rs_hist_all) and a small kernel turns those counts into each digit's
// global start (k_rs_scan_all).  Then one kernel per 8-bit pass
// (k_rs_onesweep): a CTA takes the next tile of 4096 items (an atomic tile
// counter, so tiles start in order), ranks every item inside the tile (warp
// multi-split with __match_any_sync, warps in tile order), publishes its digit
// counts, and finds the count of every digit in all earlier tiles by looking
// back over their published counts (decoupled look-back, after Merrill and
// Garland's single-pass prefix scan: a tile that has its inclusive prefix
// publishes it, so a look-back stops at the first such tile); then a
// shared-memory reorder and coalesced runs to the global positions.  Every
// wait on an earlier tile is bounded; a wait that gives up records
// kStatusTimeout.  The number of passes (ceil((S + ib) / 8) for keys of
// S + ib bits, see ClassGeom) is known only on the device: passes beyond it
// return at once, so the launch sequence is fixed and the result lands in
// buffer (passes & 1).
#include "internal.h"

namespace dpc {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsIpt = 16;                          // items per thread
constexpr int kRsTile = kRsThreads * kRsIpt;        // 4096 items per tile
constexpr int kRsWarpItems = 32 * kRsIpt;           // 512 items per warp
constexpr int kMaxPasses = (int)kSortMaxPasses;
static_assert(kRsTile == (int)kSortTile, "tile size of the scratch formula");

constexpr unsigned long long kFlagAgg = 1ull << 62;     // the tile's own counts
constexpr unsigned long long kFlagPrefix = 2ull << 62;  // counts of this and every earlier tile
constexpr unsigned long long kFlagMask = 3ull << 62;
constexpr uint32_t kSpinLimit = 1u << 20;  // ld.acquire polls of earlier tiles before giving up

// The sort's scratch: status[ntiles][256] (u64, reused by every pass), the
// digit counts and starts of every pass [kMaxPasses][256], a tile counter per
// pass.
struct SortScratch {
  unsigned long long* status;
  uint32_t* count;
  uint32_t* start;
  uint32_t* tiles;
};

__host__ __device__ inline SortScratch sort_scratch(uint32_t* base, uint32_t ntiles) {
  SortScratch z;
  z.status = reinterpret_cast<unsigned long long*>(base);
  z.count = base + (size_t)ntiles * 256u * 2u;
  z.start = z.count + kMaxPasses * 256;
  z.tiles = z.start + kMaxPasses * 256;
  return z;
}

// Digit counts of every pass in one read of the keys.
__global__ void __launch_bounds__(kRsThreads)
k_rs_hist_all(const unsigned long long* __restrict__ keys, uint32_t n,
              const ClassGeom* __restrict__ cls, uint32_t* __restrict__ count) {
  __shared__ uint32_t cnt[kMaxPasses][256];
  const int npass = sort_passes(cls->S, cls->ib);
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += kRsThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * kRsThreads + threadIdx.x; i < n; i += gridDim.x * kRsThreads) {
    const unsigned long long k = keys[i];
    for (int p = 0; p < npass && p < kMaxPasses; ++p) atomicAdd(&cnt[p][(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += kRsThreads) {
    const uint32_t v = (&cnt[0][0])[i];
    if (v) atomicAdd(&count[i], v);
  }
}

// Exclusive scan of every pass's 256 digit counts (one CTA per pass).
__global__ void __launch_bounds__(256) k_rs_scan_all(const uint32_t* __restrict__ count,
                                                     uint32_t* __restrict__ start) {
  __shared__ uint32_t part[256];
  const int p = blockIdx.x;
  const uint32_t v = count[p * 256 + threadIdx.x];
  part[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  start[p * 256 + threadIdx.x] = part[threadIdx.x] - v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct ScatterSmem {
  unsigned long long keys[kRsTile];
  uint32_t vals[kRsTile];
  uint32_t whist[kRsWarps][256];  // per-warp digit counts, then warp prefixes
  uint32_t tstart[256];           // tile-local start of each digit
  uint32_t gbase[256];            // global start of each digit in this tile
  uint32_t tile;
};

__global__ void __launch_bounds__(kRsThreads)
k_rs_onesweep(const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
              unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
              int pass, const ClassGeom* __restrict__ cls, SortScratch z, uint32_t spin_limit) {
  if (pass >= sort_passes(cls->S, cls->ib)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
  const int shift = 8 * pass;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&S.whist[0][0])[i] = 0;
  // tiles are taken in launch order, so every earlier tile has started
  if (threadIdx.x == 0) S.tile = atomicAdd(&z.tiles[pass], 1u);
  __syncthreads();
  const uint32_t tile = S.tile;

  // pass 1: warp-local stable ranks
  const uint32_t wbase = tile * kRsTile + w * kRsWarpItems;
  unsigned long long key[kRsIpt];
  uint32_t val[kRsIpt];
  uint32_t rank[kRsIpt];
#pragma unroll
  for (int r = 0; r < kRsIpt; ++r) {
    const uint32_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? kin[i] : 0ull;
    val[r] = valid ? vin[i] : 0u;
    const uint32_t dg = (uint32_t)(key[r] >> shift) & 255u;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? dg : (256u + lane)) & vmask;
    uint32_t pre = 0;
    if (valid) pre = S.whist[w][dg];
    __syncwarp();
    if (valid && (peers & lanemask_lt) == 0) S.whist[w][dg] = pre + __popc(peers);
    __syncwarp();
    rank[r] = valid ? pre + __popc(peers & lanemask_lt) : 0xffffffffu;
  }
  __syncthreads();
  // per digit: prefix over warps (tile order), the tile's count, then the
  // count of the digit in every earlier tile (look-back)
  uint32_t my_total;
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) {
      uint32_t c = S.whist[k][d];
      S.whist[k][d] = run;
      run += c;
    }
    my_total = run;
    S.tstart[d] = run;
    unsigned long long* st = z.status + (size_t)tile * 256u + d;
    uint32_t before = 0;
    if (tile == 0) {
      st_release(st, kFlagPrefix | my_total);
    } else {
      st_release(st, kFlagAgg | my_total);
      uint32_t t = tile - 1;
      uint32_t spins = 0;
      for (;;) {
        const unsigned long long v = ld_acquire(z.status + (size_t)t * 256u + d);
        const unsigned long long f = v & kFlagMask;
        if (f == 0ull) {
          if (spins++ >= spin_limit) {
            // an earlier tile has not published in time: record it, and count
            // this digit over every earlier tile's items directly (slow but
            // exact, so the sort and everything after it stay well formed)
            set_status(cls->status, kStatusTimeout);
            before = 0;
            const uint32_t upto = tile * (uint32_t)kRsTile;  // < n: this tile exists
            for (uint32_t i = 0; i < upto; ++i)
              before += ((uint32_t)(kin[i] >> shift) & 255u) == (uint32_t)d ? 1u : 0u;
            break;
          }
          continue;
        }
        before += (uint32_t)v;
        if (f == kFlagPrefix || t == 0) break;
        --t;
      }
      st_release(st, kFlagPrefix | (before + my_total));
    }
    S.gbase[d] = z.start[pass * 256 + d] + before;
  }
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    uint32_t v = threadIdx.x >= o ? S.tstart[threadIdx.x - o] : 0u;
    __syncthreads();
    S.tstart[threadIdx.x] += v;
    __syncthreads();
  }
  S.tstart[threadIdx.x] -= my_total;  // inclusive -> exclusive (own entry only)
  __syncthreads();
  // pass 2: place every item at its tile-local sorted position
#pragma unroll
  for (int r = 0; r < kRsIpt; ++r) {
    if (rank[r] != 0xffffffffu) {
      const uint32_t dg = (uint32_t)(key[r] >> shift) & 255u;
      const uint32_t pos = S.tstart[dg] + S.whist[w][dg] + rank[r];
      if (pos < (uint32_t)kRsTile) {
        S.keys[pos] = key[r];
        S.vals[pos] = val[r];
      } else {
        set_status(cls->status, kStatusIndex);
      }
    }
  }
  __syncthreads();
  // pass 3: coalesced runs to global memory
  const uint32_t tbase = tile * kRsTile;
  const uint32_t tcount = tbase < n ? min((uint32_t)kRsTile, n - tbase) : 0u;
  for (uint32_t pos = threadIdx.x; pos < tcount; pos += kRsThreads) {
    const unsigned long long k = S.keys[pos];
    const uint32_t dg = (uint32_t)(k >> shift) & 255u;
    const uint32_t dst = S.gbase[dg] + (pos - S.tstart[dg]);
    if (dst < n) {
      kout[dst] = k;
      vout[dst] = S.vals[pos];
    } else {
      set_status(cls->status, kStatusIndex);
    }
  }
}

inline uint32_t tiles_for(uint32_t n) { return (n + kRsTile - 1) / kRsTile; }

}  // namespace

size_t sort_hist_words(uint32_t n) { return sort_hist_words_for(n); }

void sort_init() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_rs_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(ScatterSmem));
    attr_set = true;
  }
}

void launch_sort(unsigned long long* codes_a, unsigned long long* codes_b, uint32_t* ids_a,
                 uint32_t* ids_b, uint32_t n, const ClassGeom* cls, uint32_t* hist,
                 cudaStream_t st) {
  if (n == 0) return;
  const uint32_t nt = tiles_for(n);
  sort_init();
  const SortScratch z = sort_scratch(hist, nt);
  const uint32_t spin = wait_limit(kSpinLimit);
  // counts, starts and tile counters of every pass
  cudaMemsetAsync(z.count, 0, sizeof(uint32_t) * (2 * kMaxPasses * 256 + kMaxPasses), st);
  unsigned hb = nt < sm_count() * 4u ? nt : sm_count() * 4u;
  k_rs_hist_all<<<hb, kRsThreads, 0, st>>>(codes_a, n, cls, z.count);
  k_rs_scan_all<<<kMaxPasses, 256, 0, st>>>(z.count, z.start);
  unsigned long long* kb[2] = {codes_a, codes_b};
  uint32_t* vb[2] = {ids_a, ids_b};
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    const int i = pass & 1, o = (pass + 1) & 1;
    cudaMemsetAsync(z.status, 0, sizeof(unsigned long long) * 256u * nt, st);
    k_rs_onesweep<<<nt, kRsThreads, sizeof(ScatterSmem), st>>>(kb[i], vb[i], kb[o], vb[o], n, pass,
                                                               cls, z, spin);
  }
  count_launches(2 + kMaxPasses);
}

}  // namespace dpc
