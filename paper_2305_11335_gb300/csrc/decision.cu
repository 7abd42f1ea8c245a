// decision.cu -- decision-graph summaries of one cutoff (Section 3, the
// decision graph plots delta against rho; cluster centers are the points
// standing out with both large).
//
//   top-k    per instance, the k points with the largest gamma = rho * delta
//            (binary64 product; descending gamma, equal gamma by the smaller
//            id; points whose product is NaN -- skipped points -- or negative
//            excluded).  One CTA per
//            instance: a radix select over the gamma bit patterns (gamma >= 0,
//            so its IEEE bits order like the values; +inf for the top point
//            is the largest) finds the k-th largest value T, a second select
//            over the ids picks the smallest ids among the points at T, and
//            the k winners are sorted in shared memory (bitonic).
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

// gamma of one point as an order-preserving bit pattern; false for a point
// that takes no part (NaN delta, or a product that is NaN or negative).
__device__ __forceinline__ bool gamma_bits(int32_t rho, double delta, unsigned long long& gb) {
  const double g = __dmul_rn((double)rho, delta);
  if (!(g >= 0.0)) return false;
  gb = g == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(g);  // -0 as +0
  return true;
}

// One CTA per instance (grid-stride over instances).
__global__ void __launch_bounds__(kDgThreads)
k_topk(const int32_t* __restrict__ rho, const double* __restrict__ delta, ClassView cv, int k,
       int32_t* __restrict__ top, double* __restrict__ gamma_out) {
  __shared__ uint32_t hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ uint32_t s_need, s_above, s_fill;
  __shared__ unsigned long long s_key[kMaxTopK];  // (gamma bits) for the sort
  __shared__ uint32_t s_id[kMaxTopK];
  const int tid = threadIdx.x;
  for (uint32_t inst = blockIdx.x; inst < cv.ninst; inst += gridDim.x) {
    const InstDev I = cv.instance(inst);
    const uint64_t base = I.out;
    const uint32_t n = I.n;
    // 1. k-th largest gamma bit pattern T (8 digits of 8 bits, high to low)
    if (tid == 0) {
      s_prefix = 0;
      s_mask = 0;
      s_need = (uint32_t)k;
      s_above = 0;
    }
    __syncthreads();
    for (int dg = 7; dg >= 0; --dg) {
      for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      const unsigned long long prefix = s_prefix, mask = s_mask;
      for (uint32_t i = tid; i < n; i += blockDim.x) {
        unsigned long long gb;
        if (!gamma_bits(rho[base + i], delta[base + i], gb)) continue;
        if ((gb & mask) == prefix) atomicAdd(&hist[(gb >> (8 * dg)) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t need = s_need, cum = 0;
        int D = -1;
        for (int b = 255; b >= 0; --b) {
          if (cum + hist[b] >= need) {
            D = b;
            break;
          }
          cum += hist[b];
        }
        if (D < 0) {  // fewer than k valid points: take them all
          s_need = 0;
          D = 0;
          s_mask = ~0ull;
          s_prefix = 0;
          s_above = 0xffffffffu;  // marker: every valid point qualifies
        } else {
          s_prefix = prefix | ((unsigned long long)D << (8 * dg));
          s_mask = mask | (255ull << (8 * dg));
          s_need = need - cum;
        }
      }
      __syncthreads();
      if (s_above == 0xffffffffu) break;
    }
    const bool all = s_above == 0xffffffffu;
    const unsigned long long T = s_prefix;
    uint32_t ties = s_need;  // points at T to take (smallest ids)
    // 2. the id threshold among the points at T: the ties-th smallest id
    uint32_t id_lim = 0xffffffffu;
    if (!all && ties > 0) {
      __shared__ uint32_t s_idp, s_idm, s_idneed;
      if (tid == 0) {
        s_idp = 0;
        s_idm = 0;
        s_idneed = ties;
      }
      __syncthreads();
      for (int dg = 3; dg >= 0; --dg) {
        for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t p = s_idp, m = s_idm;
        for (uint32_t i = tid; i < n; i += blockDim.x) {
          unsigned long long gb;
          if (!gamma_bits(rho[base + i], delta[base + i], gb) || gb != T) continue;
          if ((i & m) == p) atomicAdd(&hist[(i >> (8 * dg)) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
          uint32_t need = s_idneed, cum = 0;
          int D = 255;
          for (int b = 0; b < 256; ++b) {
            if (cum + hist[b] >= need) {
              D = b;
              break;
            }
            cum += hist[b];
          }
          s_idp = p | ((uint32_t)D << (8 * dg));
          s_idm = m | (255u << (8 * dg));
          s_idneed = need - cum;
        }
        __syncthreads();
      }
      id_lim = s_idp;  // ids <= id_lim at T are taken
    }
    // 3. gather the winners
    if (tid == 0) s_fill = 0;
    __syncthreads();
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      unsigned long long gb;
      if (!gamma_bits(rho[base + i], delta[base + i], gb)) continue;
      const bool take = all || gb > T || (gb == T && ties > 0 && i <= id_lim);
      if (take) {
        const uint32_t slot = atomicAdd(&s_fill, 1u);
        if (slot < (uint32_t)k) {
          s_key[slot] = gb;
          s_id[slot] = i;
        }
      }
    }
    __syncthreads();
    const uint32_t filled = min(s_fill, (uint32_t)k);
    // 4. bitonic sort of the winners: gamma descending, id ascending
    uint32_t P = 1;
    while (P < filled) P <<= 1;
    for (uint32_t i = filled + tid; i < P; i += blockDim.x) {
      s_key[i] = 0;
      s_id[i] = 0xffffffffu;  // padding sorts last
    }
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t i = tid; i < P; i += blockDim.x) {
          const uint32_t j = i ^ stride;
          if (j > i) {
            const bool up = (i & size) == 0;  // this half sorts "before" order
            // "before": larger gamma, then smaller id
            const bool i_before_j =
                s_key[i] > s_key[j] || (s_key[i] == s_key[j] && s_id[i] < s_id[j]);
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

__global__ void k_decision_hist(const int32_t* __restrict__ rho, const double* __restrict__ delta,
                                ClassView cv, int rho_bins, int delta_bins, double delta_lo,
                                unsigned long long* __restrict__ hist) {
  const uint64_t total = (uint64_t)cv.nchunk * 32u;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t inst, p0, end;
    cv.chunk((uint32_t)(e >> 5), inst, p0, end);
    const uint32_t p = p0 + (uint32_t)(e & 31u);
    if (p >= end) continue;
    const InstDev I = cv.instance(inst);
    const uint64_t gi = I.out + (p - I.start);
    const int32_t r = rho[gi];
    const double dl = delta[gi];
    if (dl != dl || r < 1) continue;
    int a = 31 - __clz(r);
    a = a < rho_bins ? a : rho_bins - 1;
    int b;
    if (!(dl > delta_lo)) {
      b = 0;
    } else {
      const double q = __ddiv_rn(dl, delta_lo);
      b = isinf(q) ? delta_bins - 1 : ilogb(q);
      b = b < 0 ? 0 : (b < delta_bins ? b : delta_bins - 1);
    }
    atomicAdd(&hist[((size_t)I.row * rho_bins + a) * delta_bins + b], 1ull);
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
    if (blocks > 152u * 16u) blocks = 152u * 16u;
    k_decision_pad<<<(unsigned)blocks, 256, 0, st>>>(top, gamma, m);
    count_launches(1);
  }
  if (hist && rho_bins > 0 && delta_bins > 0)
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (size_t)n_inst * rho_bins * delta_bins, st);
}

void launch_decision(const int32_t* rho, const double* delta, const ClassView& cv, int k,
                     int32_t* top, double* gamma, int rho_bins, int delta_bins, double delta_lo,
                     unsigned long long* hist, cudaStream_t st) {
  if (k > 0 && top && gamma) {
    const unsigned grid = cv.ninst < 152u * 2u ? (cv.ninst ? cv.ninst : 1u) : 152u * 2u;
    k_topk<<<grid, kDgThreads, 0, st>>>(rho, delta, cv, k, top, gamma);
    count_launches(1);
  }
  if (hist && rho_bins > 0 && delta_bins > 0) {
    uint64_t blocks = ((uint64_t)cv.nchunk * 32u + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152u * 16u) blocks = 152u * 16u;
    k_decision_hist<<<(unsigned)blocks, 256, 0, st>>>(rho, delta, cv, rho_bins, delta_bins, delta_lo,
                                                      hist);
    count_launches(1);
  }
}

int decision_max_topk() { return kMaxTopK; }

}  // namespace dpc
