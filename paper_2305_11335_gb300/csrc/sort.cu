// sort.cu -- LSD radix sort of (64-bit code, 32-bit id) pairs by code.
//
// The radix-sort primitive of Section 3.2, used here to put the points in
// Morton order.  Each 8-bit pass has three kernels:
//   hist    per-tile digit counts, written digit-major [256][ntiles]
//   scan    per digit, an exclusive scan over tiles + the digit total
//   scatter stable rank of every item inside its tile (warp multi-split with
//           __match_any_sync, warps in tile order), a shared-memory reorder,
//           then coalesced runs to the global position
// The number of passes (ceil((S + ib) / 8) for keys of S + ib bits, see
// ClassGeom) is known only on the device: passes beyond it return at once,
// so the launch sequence is fixed and the result lands in buffer
// (passes & 1).
#include "internal.h"

namespace dpc {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsIpt = 16;                          // items per thread
constexpr int kRsTile = kRsThreads * kRsIpt;        // 4096 items per tile
constexpr int kRsWarpItems = 32 * kRsIpt;           // 512 items per warp
constexpr int kMaxPasses = 8;

__global__ void __launch_bounds__(kRsThreads)
k_rs_hist(const unsigned long long* __restrict__ keys, uint32_t n, int pass,
          const ClassGeom* __restrict__ cls, uint32_t* __restrict__ hist, uint32_t ntiles) {
  if (pass >= sort_passes(cls->S, cls->ib)) return;
  __shared__ uint32_t cnt[kRsWarps][256];
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const int shift = 8 * pass;
  const int w = threadIdx.x >> 5;
  const uint32_t base = blockIdx.x * kRsTile;
#pragma unroll 4
  for (int r = 0; r < kRsIpt; ++r) {
    uint32_t i = base + r * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[w][(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kRsThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) s += cnt[k][d];
    hist[(size_t)d * ntiles + blockIdx.x] = s;
  }
}

// One block per digit: exclusive scan of that digit's per-tile counts; the
// digit total goes to hist[256 * ntiles + digit].
__global__ void __launch_bounds__(kRsThreads)
k_rs_scan(uint32_t* __restrict__ hist, uint32_t ntiles, int pass, const ClassGeom* __restrict__ cls) {
  if (pass >= sort_passes(cls->S, cls->ib)) return;
  __shared__ uint32_t part[kRsThreads];
  const int d = blockIdx.x;
  uint32_t* row = hist + (size_t)d * ntiles;
  const uint32_t per = (ntiles + kRsThreads - 1) / kRsThreads;
  const uint32_t lo = threadIdx.x * per;
  const uint32_t hi = min(lo + per, ntiles);
  uint32_t s = 0;
  for (uint32_t t = lo; t < hi; ++t) s += row[t];
  part[threadIdx.x] = s;
  __syncthreads();
  // inclusive scan of the per-thread sums (Hillis-Steele)
  for (int o = 1; o < kRsThreads; o <<= 1) {
    uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;  // exclusive
  for (uint32_t t = lo; t < hi; ++t) {
    uint32_t c = row[t];
    row[t] = run;
    run += c;
  }
  if (threadIdx.x == kRsThreads - 1) hist[(size_t)256 * ntiles + d] = part[kRsThreads - 1];
}

struct ScatterSmem {
  unsigned long long keys[kRsTile];
  uint32_t vals[kRsTile];
  uint32_t whist[kRsWarps][256];  // per-warp digit counts, then warp prefixes
  uint32_t tstart[256];           // tile-local start of each digit
  uint32_t gbase[256];            // global start of each digit (over all tiles)
};

__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
             unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
             int pass, const ClassGeom* __restrict__ cls, const uint32_t* __restrict__ hist,
             uint32_t ntiles) {
  if (pass >= sort_passes(cls->S, cls->ib)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
  const int shift = 8 * pass;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&S.whist[0][0])[i] = 0;
  // digit base over all tiles: exclusive scan of the digit totals
  {
    const uint32_t* tot = hist + (size_t)256 * ntiles;
    uint32_t v = tot[threadIdx.x];  // kRsThreads == 256
    S.gbase[threadIdx.x] = v;
  }
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    uint32_t v = threadIdx.x >= o ? S.gbase[threadIdx.x - o] : 0u;
    __syncthreads();
    S.gbase[threadIdx.x] += v;
    __syncthreads();
  }
  {
    uint32_t incl = S.gbase[threadIdx.x];
    __syncthreads();
    S.gbase[threadIdx.x] = incl - hist[(size_t)256 * ntiles + threadIdx.x];
  }
  __syncthreads();

  // pass 1: warp-local stable ranks
  const uint32_t wbase = blockIdx.x * kRsTile + w * kRsWarpItems;
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
  // per digit: prefix over warps (tile order), then the tile-local digit start
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
  const uint32_t tbase = blockIdx.x * kRsTile;
  const uint32_t tcount = min((uint32_t)kRsTile, n - tbase);
  const uint32_t* __restrict__ toff = hist;  // scanned [digit][tile]
  for (uint32_t pos = threadIdx.x; pos < tcount; pos += kRsThreads) {
    const unsigned long long k = S.keys[pos];
    const uint32_t dg = (uint32_t)(k >> shift) & 255u;
    const uint32_t dst = S.gbase[dg] + toff[(size_t)dg * ntiles + blockIdx.x] + (pos - S.tstart[dg]);
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

size_t sort_hist_words(uint32_t n) { return (size_t)257 * (tiles_for(n) ? tiles_for(n) : 1); }

void sort_init() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  unsigned long long* kb[2] = {codes_a, codes_b};
  uint32_t* vb[2] = {ids_a, ids_b};
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    const int i = pass & 1, o = (pass + 1) & 1;
    k_rs_hist<<<nt, kRsThreads, 0, st>>>(kb[i], n, pass, cls, hist, nt);
    k_rs_scan<<<256, kRsThreads, 0, st>>>(hist, nt, pass, cls);
    k_rs_scatter<<<nt, kRsThreads, sizeof(ScatterSmem), st>>>(kb[i], vb[i], kb[o], vb[o], n, pass,
                                                              cls, hist, nt);
  }
  count_launches(3 * kMaxPasses);
}

}  // namespace dpc
