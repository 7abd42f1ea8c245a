// decision.cu -- decision-graph summaries of one cutoff (Section 3, the
// decision graph plots delta against rho; cluster centers are the points
// standing out with both large).
//
//   top-k    per instance, the k points with the largest gamma = rho * delta
//            (binary64 product; descending gamma, equal gamma by the smaller
//            id; points whose product is NaN -- skipped points -- or negative
//            excluded).  A radix select over the gamma bit patterns
//            (gamma >= 0, so its IEEE bits order like the values; +inf for
//            the top point is the largest) fixes the k-th largest value T one
//            8-bit digit per pass, every pass a histogram over all points of
//            the class (warp per 32-point chunk, one atomic per distinct
//            digit) and a pick per instance; where more points sit at T than
//            are needed, four more passes over the ids fix the tie limit; a
//            gather pass collects the k winners and one CTA per instance
//            sorts them (bitonic).
//   hist     per instance, counts over (rho bin, delta bin): rho bin
//            floor(log2 rho); delta bin floor(log2(fl64(delta / delta_lo)))
//            (the exponent of the quotient), 0 for delta <= delta_lo; both
//            clipped to the last bin (+inf delta too).
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace dpc {

namespace {

constexpr int kDgThreads = 1024;
constexpr int kMaxTopK = 1024;
constexpr unsigned kFullMask = 0xffffffffu;

// gamma of one point as an order-preserving bit pattern; false for a point
// that takes no part (NaN delta, or a product that is NaN or negative).
__device__ __forceinline__ bool gamma_bits(int32_t rho, double delta, unsigned long long& gb) {
  const double g = __dmul_rn((double)rho, delta);
  if (!(g >= 0.0)) return false;
  gb = g == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(g);  // -0 as +0
  return true;
}

// Per-instance state of the radix select.
struct DgState {
  unsigned long long prefix, mask;  // gamma bits fixed so far (T when done)
  uint32_t need;    // points still to take among those matching prefix/mask
  uint32_t all;     // 1: fewer than k valid points, every valid point is taken
  uint32_t idp, idm;  // id digits fixed so far (the tie break among gamma == T)
  uint32_t idneed;  // ties still to take among ids matching idp/idm
  uint32_t tie;     // 0: every point at T is taken; 1: ids below the limit only
  uint32_t fill;    // winners gathered
  uint32_t pad;
};

__global__ void k_dg_init(DgState* __restrict__ st, uint32_t* __restrict__ hist, uint32_t ninst, int k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
    DgState z;
    z.prefix = z.mask = 0ull;
    z.need = (uint32_t)k;
    z.all = 0u;
    z.idp = z.idm = 0u;
    z.idneed = 0u;
    z.tie = 0u;
    z.fill = 0u;
    z.pad = 0u;
    st[i] = z;
  }
  const uint64_t nh = (uint64_t)ninst * 256u;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nh; e += (uint64_t)gridDim.x * blockDim.x)
    hist[e] = 0u;
}

// The CTA's share of a class: a contiguous range of chunks, and the instances
// of its first and last chunk (the only ones that can span other CTAs).
struct ChunkRange {
  uint32_t c0, c1, first, last;
};

__device__ __forceinline__ ChunkRange chunk_range(const ClassView& cv) {
  const uint32_t per = (cv.nchunk + gridDim.x - 1) / gridDim.x;
  ChunkRange r;
  r.c0 = min(cv.nchunk, blockIdx.x * per);
  r.c1 = min(cv.nchunk, r.c0 + per);
  uint32_t p0, end;
  r.first = r.last = 0xffffffffu;
  if (r.c0 < r.c1) {
    cv.chunk(r.c0, r.first, p0, end);
    cv.chunk(r.c1 - 1, r.last, p0, end);
  }
  return r;
}

// Digit histogram of one pass, warp per 32-point chunk (one instance).  The
// CTA's first and last instances count in shared memory (one global add per
// bin at the end), the instances wholly inside its range count with one
// global atomic per distinct digit of a warp.  IDS = false: gamma digit dg of
// the points matching the instance's prefix; IDS = true: id digit dg of the
// points at gamma == T matching the id prefix.
template <bool IDS>
__global__ void __launch_bounds__(256)
k_dg_hist(const int32_t* __restrict__ rho, const double* __restrict__ delta, ClassView cv,
          const DgState* __restrict__ st, uint32_t* __restrict__ hist, int dg) {
  __shared__ uint32_t sh[2][256];
  const int lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < 512; e += blockDim.x) (&sh[0][0])[e] = 0u;
  const ChunkRange R = chunk_range(cv);
  __syncthreads();
  for (uint32_t c = R.c0 + (threadIdx.x >> 5); c < R.c1; c += blockDim.x >> 5) {
    uint32_t inst, p0, end;
    cv.chunk(c, inst, p0, end);
    const DgState S = st[inst];
    if (S.all || (IDS && !S.tie)) continue;  // warp-uniform
    const InstDev I = cv.instance(inst);
    const uint32_t p = p0 + lane;
    uint32_t digit = 256u + lane;  // no digit: a key no other lane has
    if (p < end) {
      const uint32_t id = p - I.start;
      const uint64_t gi = I.out + id;
      unsigned long long gb;
      if (gamma_bits(rho[gi], delta[gi], gb)) {
        if (!IDS) {
          if ((gb & S.mask) == S.prefix) digit = (uint32_t)(gb >> (8 * dg)) & 255u;
        } else if (gb == S.prefix && (id & S.idm) == S.idp) {
          digit = (id >> (8 * dg)) & 255u;
        }
      }
    }
    const uint32_t peers = __match_any_sync(kFullMask, digit);
    if (digit < 256u && (peers & ((1u << lane) - 1u)) == 0u) {
      const uint32_t v = (uint32_t)__popc(peers);
      if (inst == R.first) atomicAdd(&sh[0][digit], v);
      else if (inst == R.last) atomicAdd(&sh[1][digit], v);
      else atomicAdd(&hist[(size_t)inst * 256u + digit], v);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 512; e += blockDim.x) {
    const uint32_t v = (&sh[0][0])[e];
    const uint32_t inst = e < 256 ? R.first : R.last;
    if (v) atomicAdd(&hist[(size_t)inst * 256u + (e & 255)], v);
  }
}

// One warp per instance: fix digit dg from the histogram, then clear it.
template <bool IDS>
__global__ void k_dg_pick(DgState* __restrict__ st, uint32_t* __restrict__ hist, uint32_t ninst, int dg) {
  const int lane = threadIdx.x & 31;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); inst < ninst; inst += nw) {
    DgState S = st[inst];
    uint32_t* h = hist + (size_t)inst * 256u;
    const bool active = !(S.all || (IDS && !S.tie));
    if (active) {
      // gamma: digits from the top (lane 0 holds 255..248); ids: from the bottom
      uint32_t c[8];
      uint32_t sum = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int b = IDS ? lane * 8 + j : 255 - (lane * 8 + j);
        c[j] = h[b];
        sum += c[j];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += t;
      }
      const uint32_t total = __shfl_sync(kFullMask, incl, 31);
      const uint32_t need = IDS ? S.idneed : S.need;
      // the digit where the running count reaches `need`
      uint32_t before = incl - sum;
      int found = -1;
      uint32_t below = 0, at = 0;
      if (before < need && incl >= need) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (found < 0 && before + c[j] >= need) {
            found = IDS ? lane * 8 + j : 255 - (lane * 8 + j);
            below = before;
            at = c[j];
          }
          if (found < 0) before += c[j];
        }
      }
      const unsigned owner = __ballot_sync(kFullMask, found >= 0);
      if (owner == 0u) {
        // fewer than `need` points match: only possible on the first gamma
        // digit (every valid point is counted there) -- take them all
        if (!IDS && lane == 0) S.all = 1u;
      } else {
        const int src = __ffs(owner) - 1;
        const int D = __shfl_sync(kFullMask, found, src);
        const uint32_t bl = __shfl_sync(kFullMask, below, src);
        const uint32_t cnt_at = __shfl_sync(kFullMask, at, src);
        if (!IDS) {
          S.prefix |= (unsigned long long)D << (8 * dg);
          S.mask |= 255ull << (8 * dg);
          S.need = need - bl;
          if (dg == 0) {  // T is fixed: S.need points at T remain to take
            S.tie = cnt_at > S.need ? 1u : 0u;
            S.idneed = S.need;
          }
        } else {
          S.idp |= (uint32_t)D << (8 * dg);
          S.idm |= 255u << (8 * dg);
          S.idneed = need - bl;
        }
      }
      (void)total;
    }
    __syncwarp();
    if (lane == 0) st[inst] = S;
#pragma unroll
    for (int j = 0; j < 8; ++j) h[lane * 8 + j] = 0u;
  }
}

// The winners of every instance into cand[inst][0..k): gamma above T, or at
// T with an id no larger than the tie limit.
__global__ void k_dg_gather(const int32_t* __restrict__ rho, const double* __restrict__ delta, ClassView cv,
                            DgState* __restrict__ st, int k, unsigned long long* __restrict__ cand_key,
                            uint32_t* __restrict__ cand_id) {
  const int lane = threadIdx.x & 31;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < cv.nchunk; c += nw) {
    uint32_t inst, p0, end;
    cv.chunk(c, inst, p0, end);
    const DgState S = st[inst];
    const InstDev I = cv.instance(inst);
    const uint32_t p = p0 + lane;
    bool take = false;
    unsigned long long gb = 0ull;
    uint32_t id = 0u;
    if (p < end) {
      id = p - I.start;
      const uint64_t gi = I.out + id;
      if (gamma_bits(rho[gi], delta[gi], gb))
        take = S.all || gb > S.prefix || (gb == S.prefix && (!S.tie || id <= S.idp));
    }
    const unsigned m = __ballot_sync(kFullMask, take);
    if (m == 0u) continue;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&st[inst].fill, (uint32_t)__popc(m));
    base = __shfl_sync(kFullMask, base, 0);
    if (take) {
      const uint32_t slot = base + __popc(m & ((1u << lane) - 1u));
      if (slot < (uint32_t)k) {
        cand_key[(size_t)inst * k + slot] = gb;
        cand_id[(size_t)inst * k + slot] = id;
      }
    }
  }
}

// One CTA per instance: bitonic sort of its winners (gamma descending, id
// ascending) into its output row.
__global__ void __launch_bounds__(kDgThreads)
k_dg_sort(ClassView cv, const DgState* __restrict__ st, int k, const unsigned long long* __restrict__ cand_key,
          const uint32_t* __restrict__ cand_id, int32_t* __restrict__ top, double* __restrict__ gamma_out) {
  __shared__ unsigned long long s_key[kMaxTopK];
  __shared__ uint32_t s_id[kMaxTopK];
  const int tid = threadIdx.x;
  for (uint32_t inst = blockIdx.x; inst < cv.ninst; inst += gridDim.x) {
    const InstDev I = cv.instance(inst);
    const uint32_t filled = min(st[inst].fill, (uint32_t)k);
    uint32_t P = 1;
    while (P < filled) P <<= 1;
    for (uint32_t i = tid; i < P; i += blockDim.x) {
      if (i < filled) {
        s_key[i] = cand_key[(size_t)inst * k + i];
        s_id[i] = cand_id[(size_t)inst * k + i];
      } else {
        s_key[i] = 0ull;
        s_id[i] = 0xffffffffu;  // padding sorts last
      }
    }
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < P; i += blockDim.x) {
          const uint32_t j = i ^ stride;
          if (j > i) {
            const bool up = (i & size) == 0;
            const bool i_before_j = s_key[i] > s_key[j] || (s_key[i] == s_key[j] && s_id[i] < s_id[j]);
            if (up != i_before_j) {
              const unsigned long long tk = s_key[i];
              s_key[i] = s_key[j];
              s_key[j] = tk;
              const uint32_t ti = s_id[i];
              s_id[i] = s_id[j];
              s_id[j] = ti;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = tid; i < k; i += blockDim.x) {
      const size_t o = (size_t)I.row * k + i;
      if ((uint32_t)i < filled) {
        top[o] = (int32_t)s_id[i];
        gamma_out[o] = __longlong_as_double((long long)s_key[i]);
      } else {
        top[o] = -1;
        gamma_out[o] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: no point
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool dg_bins(int32_t r, double dl, int rho_bins, int delta_bins,
                                        double delta_lo, int& a, int& b) {
  if (dl != dl || r < 1) return false;
  a = 31 - __clz(r);
  a = a < rho_bins ? a : rho_bins - 1;
  if (!(dl > delta_lo)) {
    b = 0;
  } else {
    const double q = __ddiv_rn(dl, delta_lo);
    b = isinf(q) ? delta_bins - 1 : ilogb(q);
    b = b < 0 ? 0 : (b < delta_bins ? b : delta_bins - 1);
  }
  return true;
}

constexpr int kHistSmemBins = 4096;  // per instance slot: 2 x 16 KB of shared memory

// Warp per chunk over the CTA's range; with SMEM the first and last instances
// of the range count in shared memory, flushed at the end.
template <bool SMEM>
__global__ void __launch_bounds__(256)
k_decision_hist(const int32_t* __restrict__ rho, const double* __restrict__ delta, ClassView cv,
                int rho_bins, int delta_bins, double delta_lo, unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[SMEM ? 2 * kHistSmemBins : 1];
  const int nb = rho_bins * delta_bins;
  const int lane = threadIdx.x & 31;
  if (SMEM)
    for (int e = threadIdx.x; e < 2 * nb; e += blockDim.x) sh[e] = 0u;
  const ChunkRange R = chunk_range(cv);
  __syncthreads();
  for (uint32_t c = R.c0 + (threadIdx.x >> 5); c < R.c1; c += blockDim.x >> 5) {
    uint32_t inst, p0, end;
    cv.chunk(c, inst, p0, end);
    const InstDev I = cv.instance(inst);
    const uint32_t p = p0 + lane;
    int a = 0, b = 0;
    bool ok = false;
    if (p < end) {
      const uint64_t gi = I.out + (p - I.start);
      ok = dg_bins(rho[gi], delta[gi], rho_bins, delta_bins, delta_lo, a, b);
    }
    const int bin = ok ? a * delta_bins + b : -1 - lane;
    const uint32_t peers = __match_any_sync(kFullMask, bin);
    if (ok && (peers & ((1u << lane) - 1u)) == 0u) {
      const uint32_t v = (uint32_t)__popc(peers);
      if (SMEM && inst == R.first) atomicAdd(&sh[bin], v);
      else if (SMEM && inst == R.last) atomicAdd(&sh[nb + bin], v);
      else atomicAdd(&hist[(size_t)I.row * nb + bin], (unsigned long long)v);
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * nb; e += blockDim.x) {
      const uint32_t v = sh[e];
      if (!v) continue;
      const uint32_t inst = e < nb ? R.first : R.last;
      const InstDev I = cv.instance(inst);
      atomicAdd(&hist[(size_t)I.row * nb + (e < nb ? e : e - nb)], (unsigned long long)v);
    }
  }
}

// Every top-k row: no point (-1, NaN) until the instance's CTA fills it.
__global__ void k_decision_pad(int32_t* top, double* gamma, size_t m) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    top[i] = -1;
    gamma[i] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

void launch_decision_init(int n_inst, int k, int32_t* top, double* gamma, int rho_bins,
                          int delta_bins, unsigned long long* hist, cudaStream_t st) {
  if (k > 0 && top && gamma) {
    const size_t m = (size_t)n_inst * k;
    uint64_t blocks = (m + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > sm_count() * 16u) blocks = sm_count() * 16u;
    k_decision_pad<<<(unsigned)blocks, 256, 0, st>>>(top, gamma, m);
    count_launches(1);
  }
  if (hist && rho_bins > 0 && delta_bins > 0)
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (size_t)n_inst * rho_bins * delta_bins, st);
}

size_t decision_scratch_bytes(uint32_t ninst, int k) {
  const size_t a = ((sizeof(DgState) * ninst + 255) / 256) * 256;
  const size_t h = ((sizeof(uint32_t) * 256u * ninst + 255) / 256) * 256;
  const size_t c = ((sizeof(unsigned long long) * (size_t)ninst * k + 255) / 256) * 256;
  const size_t d = ((sizeof(uint32_t) * (size_t)ninst * k + 255) / 256) * 256;
  return a + h + c + d;
}

void launch_decision(const int32_t* rho, const double* delta, const ClassView& cv, int k,
                     int32_t* top, double* gamma, int rho_bins, int delta_bins, double delta_lo,
                     unsigned long long* hist, void* scratch, cudaStream_t st) {
  if (k > 0 && top && gamma && cv.ninst > 0) {
    char* b = (char*)scratch;
    const size_t a = ((sizeof(DgState) * cv.ninst + 255) / 256) * 256;
    const size_t h = ((sizeof(uint32_t) * 256u * cv.ninst + 255) / 256) * 256;
    const size_t c = ((sizeof(unsigned long long) * (size_t)cv.ninst * k + 255) / 256) * 256;
    DgState* S = (DgState*)b;
    uint32_t* H = (uint32_t*)(b + a);
    unsigned long long* ck = (unsigned long long*)(b + a + h);
    uint32_t* ci = (uint32_t*)(b + a + h + c);
    uint64_t cb = ((uint64_t)cv.nchunk + 31) / 32;  // at least 32 chunks per CTA
    const unsigned chunk_blocks = (unsigned)(cb < 1 ? 1 : (cb > sm_count() * 8u ? sm_count() * 8u : cb));
    uint64_t ib = ((uint64_t)cv.ninst + 7) / 8;
    const unsigned inst_blocks = (unsigned)(ib < 1 ? 1 : (ib > sm_count() * 16u ? sm_count() * 16u : ib));
    k_dg_init<<<inst_blocks, 256, 0, st>>>(S, H, cv.ninst, k);
    for (int dg = 7; dg >= 0; --dg) {
      k_dg_hist<false><<<chunk_blocks, 256, 0, st>>>(rho, delta, cv, S, H, dg);
      k_dg_pick<false><<<inst_blocks, 256, 0, st>>>(S, H, cv.ninst, dg);
    }
    for (int dg = 3; dg >= 0; --dg) {
      k_dg_hist<true><<<chunk_blocks, 256, 0, st>>>(rho, delta, cv, S, H, dg);
      k_dg_pick<true><<<inst_blocks, 256, 0, st>>>(S, H, cv.ninst, dg);
    }
    k_dg_gather<<<chunk_blocks, 256, 0, st>>>(rho, delta, cv, S, k, ck, ci);
    const unsigned grid = cv.ninst < sm_count() * 2u ? cv.ninst : sm_count() * 2u;
    k_dg_sort<<<grid, kDgThreads, 0, st>>>(cv, S, k, ck, ci, top, gamma);
    count_launches(1 + 2 * 12 + 2);
  }
  if (hist && rho_bins > 0 && delta_bins > 0) {
    uint64_t blocks = ((uint64_t)cv.nchunk + 31) / 32;  // at least 32 chunks per CTA
    if (blocks < 1) blocks = 1;
    if (blocks > sm_count() * 8u) blocks = sm_count() * 8u;
    if (rho_bins * delta_bins <= kHistSmemBins)
      k_decision_hist<true><<<(unsigned)blocks, 256, 0, st>>>(rho, delta, cv, rho_bins, delta_bins,
                                                              delta_lo, hist);
    else
      k_decision_hist<false><<<(unsigned)blocks, 256, 0, st>>>(rho, delta, cv, rho_bins, delta_bins,
                                                               delta_lo, hist);
    count_launches(1);
  }
}

int decision_max_topk() { return kMaxTopK; }

}  // namespace dpc
