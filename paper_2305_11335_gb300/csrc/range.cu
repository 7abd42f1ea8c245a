// range.cu -- priority range search (the appendix on range queries): for a
// query (instance, closed axis-parallel box [lo, hi], threshold rho_q), every
// point of the instance inside the box whose priority -- its density -- is
// above rho_q.
//
// The search runs on the class's radix tree after the bottom-up pass: a node
// is entered only if its largest key says some point below it has
// rho > rho_q and its bounding box meets the query box, which is the pruning
// the appendix describes for the priority search kd-tree (the nodes with a
// large enough key form an upper part of the tree, and the search is a plain
// range search on that part).  One warp per query: a shared-memory stack of
// internal nodes, up to 32 popped per step (one per lane); a lane whose
// pushes find the stack full walks that subtree alone with the parent links
// (no stack).  The sorted float copy holds every coordinate exactly (float32
// inputs as they are, int32 inputs are range-checked to |x| <= 2^24), so both
// the box tests and the node tests are exact.
//
// Two passes per class: COUNT writes each query's number of matches; FILL
// writes (query << 31 | instance-local id) for every match at the query's
// offset.  The host sorts those keys (radix sort) and a last kernel scatters
// the first max_out ids of every query, ascending, into its output row.
#include <cstdint>

#include "internal.h"

namespace dpc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPrThreads = 128;
constexpr int kPrWarps = kPrThreads / 32;
constexpr int kPrStack = 2048;  // internal nodes per warp

template <int DP>
struct PrQuery {
  double lo[DP], hi[DP];  // the instance's d <= DP coordinates are tested
  int32_t rq;
  int d;
};

template <int DP>
__device__ __forceinline__ bool point_in(const float* __restrict__ spts, uint32_t t,
                                         const PrQuery<DP>& Q) {
  const Pt<DP> p = load_pt<DP>(spts, t);
  bool ok = true;
#pragma unroll
  for (int a = 0; a < DP; ++a)
    if (a < Q.d) ok &= (double)p.x[a] >= Q.lo[a] && (double)p.x[a] <= Q.hi[a];
  return ok;
}

__device__ __forceinline__ int32_t key_rho(unsigned long long k) { return (int32_t)(k >> 32); }

// Child test from its parent's record: some key below is above the
// threshold, and the box meets.
template <int DP>
__device__ __forceinline__ bool child_ok(const ChildRec<DP>& r, int s, const PrQuery<DP>& Q) {
  if (key_rho(r.key[s]) <= Q.rq) return false;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < DP; ++a)
    if (a < Q.d) ok &= (double)r.hi[s][a] >= Q.lo[a] && (double)r.lo[s][a] <= Q.hi[a];
  return ok;
}

// Leaf test; a match goes to `hit(t)`.
template <int DP, typename Hit>
__device__ __forceinline__ void leaf(const float* __restrict__ spts,
                                     const unsigned long long* __restrict__ skey, uint32_t t,
                                     uint32_t n, const PrQuery<DP>& Q, bool& bad, Hit&& hit) {
  if (t >= n) {
    bad = true;
    return;
  }
  if (key_rho(skey[t]) > Q.rq && point_in<DP>(spts, t, Q)) hit(t);
}

// One lane alone over the subtree of internal node r (r already tested),
// following parent links instead of a stack; false if it gave up.
template <int DP, typename Hit>
__device__ bool walk_alone(const Node* __restrict__ nodes, const float* __restrict__ nbox,
                           const float* __restrict__ spts, const unsigned long long* __restrict__ skey,
                           uint32_t n, uint32_t r, const PrQuery<DP>& Q, bool& bad, Hit&& hit) {
  uint32_t cur = r;
  bool down = true;
  const uint64_t limit = 4ull * n + 64ull;
  for (uint64_t it = 0; it < limit; ++it) {
    if (cur + 1 >= n) {
      bad = true;
      return false;
    }
    if (down) {
      const ChildRec<DP> rc = load_rec<DP>(nbox, cur);
      const uint32_t l = rc.child[0], rr = rc.child[1];
      if (l & kLeafBit) leaf<DP>(spts, skey, l & ~kLeafBit, n, Q, bad, hit);
      if (rr & kLeafBit) leaf<DP>(spts, skey, rr & ~kLeafBit, n, Q, bad, hit);
      if (!(l & kLeafBit) && child_ok<DP>(rc, 0, Q)) {
        cur = l;
        continue;
      }
      if (!(rr & kLeafBit) && child_ok<DP>(rc, 1, Q)) {
        cur = rr;
        continue;
      }
      down = false;
    }
    // climbing: cur's subtree is done
    if (cur == r) return true;
    const uint32_t p = nodes[cur].parent;
    if (p + 1 >= n) {
      bad = true;
      return false;
    }
    const ChildRec<DP> rp = load_rec<DP>(nbox, p);
    const uint32_t pr = rp.child[1];
    if (rp.child[0] == cur && !(pr & kLeafBit) && child_ok<DP>(rp, 1, Q)) {
      cur = pr;
      down = true;
      continue;
    }
    cur = p;
  }
  bad = true;
  return false;
}

// FILL = false: count[q] (and cnt[q], the count restricted to this class).
// FILL = true: keys at off[q] + (the warp's running position).
template <int DP, bool FILL>
__global__ void __launch_bounds__(kPrThreads)
k_prange(const float* __restrict__ spts, const uint32_t* __restrict__ sid,
         const unsigned long long* __restrict__ skey, ClassView cv, const Node* __restrict__ nodes,
         const float* __restrict__ nbox, const uint32_t* __restrict__ roots, uint32_t nq,
         int32_t n_inst, const int32_t* __restrict__ q_inst, const double* __restrict__ q_box,
         const int32_t* __restrict__ q_rho, const int32_t* __restrict__ rowmap, int32_t one_row,
         uint32_t* __restrict__ cnt, long long* __restrict__ count,
         const unsigned long long* __restrict__ off, unsigned long long* __restrict__ out_keys,
         int stack_cap, int* __restrict__ status) {
  __shared__ uint32_t s_stk[kPrWarps][kPrStack];
  __shared__ uint32_t s_fill[kPrWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t* stk = s_stk[wib];
  const uint32_t n = cv.N;
  bool bad = false;
  for (uint32_t q = blockIdx.x * kPrWarps + wib; q < nq; q += gridDim.x * kPrWarps) {
    const int32_t row = q_inst[q];
    int32_t loc = -1;
    if (row >= 0 && row < n_inst) loc = rowmap ? rowmap[row] : (row == one_row ? 0 : -1);
    if (loc < 0 || (uint32_t)loc >= cv.ninst) {
      if (!FILL && lane == 0) cnt[q] = 0u;  // another class's query (or a bad row, flagged once)
      continue;
    }
    const InstDev I = cv.instance((uint32_t)loc);
    PrQuery<DP> Q;
    Q.d = I.d;
    Q.rq = q_rho[q];
#pragma unroll
    for (int a = 0; a < DP; ++a) {
      Q.lo[a] = q_box[(size_t)q * 2 * kMaxDim + a];
      Q.hi[a] = q_box[(size_t)q * 2 * kMaxDim + kMaxDim + a];
    }
    const uint64_t base = FILL ? off[q] : 0ull;
    const uint32_t cap = FILL ? cnt[q] : 0u;  // FILL: the count pass's number
    uint32_t mine = 0;  // COUNT: this lane's matches
    if (lane == 0) s_fill[wib] = 0u;
    __syncwarp();
    auto hit = [&](uint32_t t) {
      if constexpr (FILL) {
        const uint32_t slot = atomicAdd(&s_fill[wib], 1u);
        const uint32_t id = sid[t] - (uint32_t)I.out;
        if (slot < cap) out_keys[base + slot] = ((unsigned long long)q << 31) | (unsigned long long)id;
        else bad = true;
      } else {
        ++mine;
      }
    };
    if (I.n == 1) {
      if (lane == 0) leaf<DP>(spts, skey, I.start, n, Q, bad, hit);
    } else if (I.n > 1) {
      const uint32_t root = roots[loc];
      bool go = false;
      if (root + 1 >= n) {
        bad = true;
      } else {
        go = true;  // the root's own key and box live in its parent's record: test its children
      }
      if (lane == 0 && go) stk[0] = root;
      int sp = go ? 1 : 0;
      __syncwarp();
      while (sp > 0) {
        const int take = sp < 32 ? sp : 32;
        const int b0 = sp - take;
        uint32_t keep[2];
        int nk = 0;
        if (lane < take) {
          const uint32_t ni = stk[b0 + lane];
          if (ni + 1 >= n) {
            bad = true;
          } else {
            const ChildRec<DP> rc = load_rec<DP>(nbox, ni);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
              const uint32_t c = rc.child[s];
              if (c & kLeafBit) {
                leaf<DP>(spts, skey, c & ~kLeafBit, n, Q, bad, hit);
              } else if (c + 1 >= n) {
                bad = true;
              } else if (child_ok<DP>(rc, s, Q)) {
                keep[nk++] = c;
              }
            }
          }
        }
        uint32_t incl = (uint32_t)nk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = (int)__shfl_sync(kFull, incl, 31);
        const int pos = b0 + (int)incl - nk;
        __syncwarp();
        for (int s = 0; s < nk; ++s) {
          if (pos + s < stack_cap) stk[pos + s] = keep[s];
          else if (!walk_alone<DP>(nodes, nbox, spts, skey, n, keep[s], Q, bad, hit)) bad = true;
        }
        sp = min(b0 + total, stack_cap);
        __syncwarp();
      }
    }
    if constexpr (!FILL) {
      uint32_t m = mine;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(kFull, m, o);
      if (lane == 0) {
        cnt[q] = m;
        count[q] = (long long)m;
      }
    }
    __syncwarp();
  }
  if (bad) set_status(status, kStatusIndex);
}

// Query checks and output defaults: count 0, rows of -1; a row index outside
// the batch is a data error.
__global__ void k_prange_init(uint32_t nq, int32_t n_inst, const int32_t* __restrict__ q_inst,
                              long long* __restrict__ count, int32_t* __restrict__ ids, int max_out,
                              int* __restrict__ status) {
  const uint64_t total = (uint64_t)nq * (uint64_t)(max_out > 0 ? max_out : 0);
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x)
    ids[e] = -1;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    count[q] = 0;
    const int32_t r = q_inst[q];
    if (r < 0 || r >= n_inst) set_status(status, kStatusQuery);
  }
}

// Exclusive scan of cnt[0..nq) into off[0..nq], one CTA (off[nq] = total).
__global__ void __launch_bounds__(1024) k_prange_scan(const uint32_t* __restrict__ cnt, uint32_t nq,
                                                      unsigned long long* __restrict__ off) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0ull;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < nq; c0 += 1024u) {
    const uint32_t i = c0 + threadIdx.x;
    const unsigned long long v = i < nq ? cnt[i] : 0ull;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const unsigned long long t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nq) off[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[nq] = carry;
}

// Sorted keys -> the first max_out ids of every query's row.
__global__ void k_prange_scatter(const unsigned long long* __restrict__ keys, uint64_t total,
                                 const unsigned long long* __restrict__ off, uint32_t nq,
                                 int max_out, int32_t* __restrict__ ids, int* __restrict__ status) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[e];
    const uint32_t q = (uint32_t)(k >> 31);
    if (q >= nq || e < off[q] || e >= off[q + 1]) {
      set_status(status, kStatusIndex);
      continue;
    }
    const uint64_t j = e - off[q];
    if (j < (uint64_t)max_out) ids[(size_t)q * max_out + j] = (int32_t)(k & 0x7fffffffull);
  }
}

inline unsigned grid_cap(uint64_t items, int per, unsigned cap) {
  uint64_t b = (items + per - 1) / per;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, bool FILL>
void prange_dp(const float* spts, const uint32_t* sid, const unsigned long long* skey,
               const ClassView& cv, const Node* nodes, const float* nbox, const uint32_t* roots,
               const PrangeArgs& a, uint32_t* cnt, const unsigned long long* off,
               unsigned long long* keys, int* status, cudaStream_t st) {
  k_prange<DP, FILL><<<grid_cap(a.nq, kPrWarps, sm_count() * 8u), kPrThreads, 0, st>>>(
      spts, sid, skey, cv, nodes, nbox, roots, a.nq, a.n_inst, a.q_inst, a.q_box, a.q_rho,
      a.rowmap, a.one_row, cnt, a.count, off, keys,
      a.stack_cap > 0 && a.stack_cap < kPrStack ? a.stack_cap : kPrStack, status);
}

}  // namespace

void launch_prange_init(const PrangeArgs& a, int32_t* ids, int max_out, int* status,
                        cudaStream_t st) {
  const uint64_t items = (uint64_t)a.nq * (uint64_t)(max_out > 0 ? max_out : 1);
  k_prange_init<<<grid_cap(items, 256, sm_count() * 16u), 256, 0, st>>>(a.nq, a.n_inst, a.q_inst, a.count,
                                                                 ids, max_out, status);
  count_launches(1);
}

void launch_prange(int dp, bool fill, const float* spts, const uint32_t* sid,
                   const unsigned long long* skey, const ClassView& cv, const Node* nodes,
                   const float* nbox, const uint32_t* roots, const PrangeArgs& a, uint32_t* cnt,
                   const unsigned long long* off, unsigned long long* keys, int* status,
                   cudaStream_t st) {
  if (a.nq == 0) return;
  if (dp == 2) {
    if (fill) prange_dp<2, true>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
    else prange_dp<2, false>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
  } else if (dp == 4) {
    if (fill) prange_dp<4, true>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
    else prange_dp<4, false>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
  } else {
    if (fill) prange_dp<8, true>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
    else prange_dp<8, false>(spts, sid, skey, cv, nodes, nbox, roots, a, cnt, off, keys, status, st);
  }
  count_launches(1);
}

void launch_prange_scan(const uint32_t* cnt, uint32_t nq, unsigned long long* off,
                        cudaStream_t st) {
  k_prange_scan<<<1, 1024, 0, st>>>(cnt, nq, off);
  count_launches(1);
}

void launch_prange_scatter(const unsigned long long* keys, uint64_t total,
                           const unsigned long long* off, uint32_t nq, int max_out, int32_t* ids,
                           int* status, cudaStream_t st) {
  if (total == 0 || max_out <= 0) return;
  k_prange_scatter<<<grid_cap(total, 256, sm_count() * 16u), 256, 0, st>>>(keys, total, off, nq, max_out,
                                                                     ids, status);
  count_launches(1);
}

}  // namespace dpc
