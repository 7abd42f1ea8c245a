// tc_density.cu -- rho_i (Definition 1) for 5- to 8-dimensional points with
// the distance tiles on the tensor cores (tcgen05, TF32 operands, FP32
// accumulation in tensor memory).
//
// Work layout: every occupied cell is cut into pieces of at most 128 of its
// points (k_tc_pieces); a CTA of 4 warps takes pieces one by one from a global
// work counter.  The 128 rows of the MMA are the piece's queries, the columns
// the candidates of the cell's block, 256 per MMA.  With the augmented rows
//     a = [q_0 .. q_7, (1 + e) |q|^2, 1, 0 ..]                 (query, M = 128)
//     b = [-2 c_0 .. -2 c_7, 1, (1 + e) |c|^2 - (1 - e) t_in, 0 ..] (N = 256)
// (e = 2^-14) one product a . b = s + E - t_in: the squared distance s, plus
// the error allowance E = e (|q|^2 + |c|^2 + t_in), minus the float32 filter's
// inner threshold, so the epilogue only compares the accumulator with 0.
// Every operand is split into a TF32 high part and a TF32 remainder and the
// three products hi.hi + hi.lo + lo.hi are accumulated (measured error ~2^-22
// relative to |a||b|); coordinates are taken relative to the piece's first
// query so the norms stay small.  Thread t owns accumulator row t (its query)
// and counts the 256 columns of each tile.
//
// Exactness: E is far above the split-TF32 error, the FP32 accumulation error
// (at most about 2^-16.4 times the same sum of norms and t_in) and the
// float32 norm rounding, so acc <= 0 proves s <= t_in, hence s64 <= d_cut^2
// (t_in, t_out as in the float32 filter); acc > W, with W = (t_out - t_in) +
// 1.25 e (|q|^2 + the largest |c|^2 of the 32 columns + t_in) (rounded up),
// proves s > t_out, hence s64 > d_cut^2.  Pairs in between are recounted
// with the canonical binary64 distance from the original coordinates, so rho
// is exactly the binary64 count.  Dense blocks only: the autotuner picks this
// layout where it is faster than the float32 layouts.
#include <cstdint>

#include "block.cuh"
#include "internal.h"

namespace dpc {

namespace {

constexpr int kTcThreads = 256;     // 8 warps: warps w and w + 4 share accumulator lanes
constexpr int kTcM = 128;            // queries per MMA (rows)
constexpr int kTcN = 256;            // candidates per MMA (columns)
constexpr int kTcK = 16;             // augmented row length: two K = 8 steps
constexpr float kTcErr = 0x1p-14f;
// one candidate row per thread: warp w stages columns 32w .. 32w + 31
static_assert(kTcN == kTcThreads, "candidate rows per thread");
constexpr float kTcFar = 1e30f;      // |c|^2 of a padding candidate: never counted
constexpr uint32_t kTcWaitLimit = 1u << 26;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// Byte offset of element (row r, k) in the K-major, non-swizzled operand
// layout of a ROWS-row operand: core matrices of 8 rows x 16 bytes; the two
// core matrices of one 8-element K step 128 bytes apart (leading offset),
// 8-row groups 256 bytes apart (stride offset), K steps ROWS * 32 bytes apart.
template <int ROWS>
__device__ __forceinline__ uint32_t op_off(int r, int k) {
  return (uint32_t)((k >> 3) * (ROWS * 32) + (r >> 3) * 256 + ((k >> 2) & 1) * 128 + (r & 7) * 16 +
                    (k & 3) * 4);
}

// Shared-memory matrix descriptor (sm_100 family): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

struct TcSmem {
  float a[2][kTcM * kTcK];      // query rows, TF32 high part / remainder
  float b[2][kTcN * kTcK];      // candidate rows
  float c[kTcN * 8];            // candidate coordinates (original)
  float cmax[kTcN / 32];        // per 32 columns (the rows one warp stages): largest |c'|^2
  int cnt[kTcM];                // per query: the two column halves' counts
  RunTable rt;
  unsigned long long mbar;
  uint32_t tmem;
  int nr;
  uint32_t item;
};

// Writes the TF32 split of the augmented row v (kTcK floats) into row r of
// operand pair ops.
template <int ROWS>
__device__ __forceinline__ void put_row(float (*ops)[ROWS * kTcK], int r, const float* v) {
#pragma unroll
  for (int k = 0; k < kTcK; ++k) {
    const float h = tf32_rna(v[k]);
    const float l = tf32_rna(v[k] - h);
    *(float*)((char*)ops[0] + op_off<ROWS>(r, k)) = h;
    *(float*)((char*)ops[1] + op_off<ROWS>(r, k)) = l;
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.b32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// The piece list: (hash slot, first point) of every 128-point piece of every
// occupied cell, from a scan of the hash table (one atomic per warp).
// Also gives every point the order key of density 0 (and rho 0) first, or,
// for the near phase, lambda = -1: a CTA that gives up on a wait (the MMA did
// not complete in time) leaves its pieces unwritten, and the later phases
// must still see one valid key per position and dependent pointers that form
// no cycle.
__global__ void k_tc_pieces(HashInfo* hi, const unsigned long long* __restrict__ hkeys,
                            const uint2* __restrict__ hvals, uint32_t n, uint2* __restrict__ pieces,
                            const uint32_t* __restrict__ sid, int32_t* __restrict__ rho_out,
                            unsigned long long* __restrict__ skey, bool init_keys,
                            int32_t* __restrict__ lambda) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t id = sid[q];
    if (init_keys) {
      rho_out[id] = 0;
      skey[q] = order_key(0, id);
    }
    if (lambda) lambda[id] = -1;  // near phase: what a CTA that gave up leaves
  }
  const uint32_t T = hi->hmask + 1;
  const int lane = threadIdx.x & 31;
  const uint32_t T_pad = (T + 31) & ~31u;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < T_pad; s += gridDim.x * blockDim.x) {
    uint2 run = make_uint2(0u, 0u);
    if (s < T && hkeys[s] != kEmpty) run = clip_run(hvals[s], n);
    const uint32_t np = (run.y - run.x + kTcM - 1) / kTcM;
    uint32_t incl = np;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    const uint32_t tot = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && tot) base = atomicAdd(&hi->npieces, tot);
    base = __shfl_sync(kFull, base, 31) + incl - np;
    for (uint32_t j = 0; j < np; ++j) pieces[base + j] = make_uint2(s, run.x + j * kTcM);
  }
}

template <int G>
__global__ void __launch_bounds__(kTcThreads)
k_density_tc(const float* __restrict__ spts, const uint32_t* __restrict__ sid, ClassView cv,
             const CutGeom* __restrict__ cuts, HashInfo* hi,
             const unsigned long long* __restrict__ hkeys, const uint2* __restrict__ hvals,
             const uint2* __restrict__ pieces, int32_t* __restrict__ rho_out,
             unsigned long long* __restrict__ skey, Counters* ctr, uint32_t poll_limit) {
  constexpr int DP = 8;
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t npieces = hi->npieces;
  const uint32_t n = cv.N;
  const uint32_t mbar = smem_addr(&sm.mbar);

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&sm.tmem)), "r"(kTcN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;
  // warp w reads accumulator lanes 32 (w % 4) .. (the rows of queries
  // 32 (w % 4) ..) and the columns of half w / 4
  const int qrow = (warp & 3) * 32 + lane;
  const int chalf = warp >> 2;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(chalf * (kTcN / 2));
  uint32_t phase = 0;
  unsigned long long band = 0, pairs = 0;
  bool stop = false;

  while (!stop) {
    if (tid == 0) sm.item = atomicAdd(&hi->work, 1u);
    __syncthreads();
    const uint32_t item = sm.item;
    __syncthreads();
    if (item >= npieces) break;
    // the piece's cell: its run of sorted points, instance, geometry and block
    const uint2 pc = pieces[item];
    const uint32_t slot = pc.x & hmask;
    const unsigned long long key = hkeys[slot];
    const uint2 run = clip_run(hvals[slot], n);
    uint32_t inst = key_inst(key, S, ib);
    if (inst >= cv.ninst) inst = 0;
    const unsigned long long code = key_code(key, S, ib);
    const CutGeom& C = cuts[inst];
    const int R = C.R;
    const int cmax = (1 << (cv.geom[inst].B - C.k)) - 1;
    const double dc2 = C.dc2;
    const float t_in = C.t_in, t_out = C.t_out;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    uint32_t c0[G];
    unmorton<G>(code, c0);
    if (warp == 0) {
      Union<G> u;
      block_union<G>(c0, R, cmax, u);
      const int nrr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, sm.rt);
      if (lane == 0) sm.nr = nrr;
    }
    __syncthreads();
    const int nr = sm.nr;
    const uint32_t total = sm.rt.pre[nr];
    if (tid == 0) {
      const uint32_t q0p = pc.y < run.x ? run.x : pc.y;
      pairs += (unsigned long long)min((uint32_t)kTcM, run.y - q0p) * total;
    }
    {
      const uint32_t q0 = pc.y < run.x ? run.x : pc.y;
      // query rows: this thread's point, relative to the piece's first point
      const uint32_t q = q0 + (uint32_t)qrow;
      const bool inq = q < run.y;
      const Pt<DP> o = load_pt<DP>(spts, q0);
      Pt<DP> me;
#pragma unroll
      for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
      if (inq) me = load_pt<DP>(spts, q);
      float nq = 0.f;
      {
        float row[kTcK];
#pragma unroll
        for (int a = 0; a < DP; ++a) {
          const float t = inq ? me.x[a] - o.x[a] : 0.f;
          row[a] = t;
          nq = fmaf(t, t, nq);
        }
        row[8] = nq * (1.f + kTcErr);
        row[9] = 1.f;
#pragma unroll
        for (int a = 10; a < kTcK; ++a) row[a] = 0.f;
        if (chalf == 0) put_row<kTcM>(sm.a, qrow, row);
      }
      if (tid < kTcM) sm.cnt[tid] = 0;
      int32_t cnt = 0;
      // This thread's candidate of the tile starting at w (row tid), loaded
      // one tile ahead: the next tile's load is issued right after this
      // tile's MMA, so it is in flight during the MMA and the epilogue.
      auto fetch = [&](uint32_t w) {
        Pt<DP> x;
#pragma unroll
        for (int a = 0; a < DP; ++a) x.x[a] = 0.f;
        const uint32_t e = w + (uint32_t)tid;
        if (e < total) {
          int lo = 0, hi2 = nr - 1;
          while (lo < hi2) {
            const int mid = (lo + hi2 + 1) >> 1;
            if (sm.rt.pre[mid] <= e) lo = mid;
            else hi2 = mid - 1;
          }
          x = load_pt<DP>(spts, sm.rt.start[lo] + (e - sm.rt.pre[lo]));
        }
        return x;
      };
      Pt<DP> xnext = fetch(0);
      for (uint32_t w0 = 0; w0 < total && !stop; w0 += kTcN) {
        // candidate rows: one per thread
#pragma unroll
        for (int h = 0; h < kTcN / kTcThreads; ++h) {
          const int r = tid + h * kTcThreads;
          const uint32_t e = w0 + (uint32_t)r;
          float row[kTcK];
          Pt<DP> x;
          float ncr = 0.f;
          if (e < total) {
            x = xnext;
            float nc = 0.f;
#pragma unroll
            for (int a = 0; a < DP; ++a) {
              const float t = x.x[a] - o.x[a];
              row[a] = -2.f * t;
              nc = fmaf(t, t, nc);
            }
            row[8] = 1.f;
            // the threshold folded in: the product is s + E - t_in
            row[9] = nc * (1.f + kTcErr) - t_in * (1.f - kTcErr);
            ncr = nc;
          } else {
#pragma unroll
            for (int a = 0; a < DP; ++a) { x.x[a] = 0.f; row[a] = 0.f; }
            row[8] = 0.f;
            row[9] = kTcFar;
          }
          {
            float m = ncr;
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
            if (lane == 0) sm.cmax[warp] = m;
          }
#pragma unroll
          for (int a = 10; a < kTcK; ++a) row[a] = 0.f;
          put_row<kTcN>(sm.b, r, row);
#pragma unroll
          for (int a = 0; a < DP; ++a) sm.c[r * DP + a] = x.x[a];
        }
        // operands written by the threads -> visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
          const uint32_t ab = smem_addr(sm.a[0]), al = smem_addr(sm.a[1]);
          const uint32_t bb = smem_addr(sm.b[0]), bl = smem_addr(sm.b[1]);
          const uint32_t as[3] = {ab, ab, al}, bs[3] = {bb, bl, bb};
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int sp = 0; sp < 3; ++sp) {
              const uint64_t ad = smem_desc(as[sp] + ks * (kTcM * 32));
              const uint64_t bd = smem_desc(bs[sp] + ks * (kTcN * 32));
              const uint32_t accum = (ks | sp) ? 1u : 0u;
              asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                           " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n"
                           :: "r"(tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum) : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(mbar) : "memory");
        }
        if (w0 + kTcN < total) xnext = fetch(w0 + kTcN);
        const bool ok = mbar_wait(mbar, phase, poll_limit);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {  // the MMA did not finish in time: record and stop
          if (tid == 0) set_status(cv.cls->status, kStatusTimeout);
          // let the MMA in flight finish (the full limit, whatever poll_limit
          // was) before tensor memory is freed and the CTA exits
          mbar_wait(mbar, phase ^ 1u, kTcWaitLimit);
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int ncol = (int)min((uint32_t)kTcN, total - w0);
        const float tw = __fsub_ru(t_out, t_in);
        for (int cl = 0; cl < kTcN / 2; cl += 32) {
          const int cb = chalf * (kTcN / 2) + cl;  // first column of this load
          if (cb >= ncol) break;  // warp-uniform
          float v[32];
          tmem_ld32(trow + (uint32_t)cl, v);
          // Above W the pair is certainly farther than t_out: (t_out - t_in)
          // plus 1.25 E at this query's norm and the largest candidate norm
          // of these 32 columns (warp cb / 32 staged them), rounded up, so
          // that acc > W implies s > t_out.
          const float W = __fadd_ru(
              tw, __fmul_ru(1.25f * kTcErr, __fadd_ru(__fadd_ru(nq, sm.cmax[cb >> 5]), t_in)));
          const uint32_t wbits = __float_as_uint(W);
          if (inq) {
            // On the bit patterns: a negative accumulator (sign bit set,
            // -0 included) is counted; one in [+0, W] (an unsigned compare,
            // W >= 0) goes to the binary64 recount, +0 included.
            unsigned ci = 0, bm = 0;  // bm: columns of this load in the band
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const uint32_t b = __float_as_uint(v[j]);
              ci += b >> 31;
              bm |= (b <= wbits) ? (1u << j) : 0u;
            }
            cnt += (int32_t)ci;
            while (bm) {  // band pairs: the canonical binary64 distance decides
              const int j = __ffs((int)bm) - 1;
              bm &= bm - 1u;
              Pt<DP> x;
#pragma unroll
              for (int a = 0; a < DP; ++a) x.x[a] = sm.c[(cb + j) * DP + a];
              ++band;
              cnt += dist64<DP>(me, x) <= dc2 ? 1 : 0;
            }
          }
        }
        // every read of the accumulator and the operands done before the next tile
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
      }
      // the two halves of each query's count
      if (inq) atomicAdd(&sm.cnt[qrow], cnt);
      __syncthreads();
      if (inq && chalf == 0 && !stop) {
        const int32_t total_cnt = sm.cnt[qrow];
        const uint32_t id = sid[q];
        rho_out[id] = total_cnt;
        skey[q] = order_key(total_cnt, id);
      }
      __syncthreads();
    }
  }
  // release the tensor memory
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcN) : "memory");
  for (int o = 16; o > 0; o >>= 1) band += __shfl_xor_sync(kFull, band, o);
  if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  if (tid == 0 && pairs) atomicAdd(&ctr->pairs, pairs);
}

// Dynamic shared memory per CTA: at least the layout, and enough that no
// more than two CTAs share an SM (each holds kTcN of the 512 tensor-memory
// columns for its whole life, so a third would wait for one to finish).
constexpr size_t kTcSmemBytes = sizeof(TcSmem) > 100 * 1024 ? sizeof(TcSmem) : 100 * 1024;
static_assert(sizeof(TcSmem) <= 200 * 1024, "shared-memory layout too large");


// ---------------------------------------------------------------------------
// The near phase of the dependent search (Definitions 2-3) on the tensor
// cores: the same pieces and tiles, with b = [-2 c', 1, |c'|^2] so that the
// accumulator is s itself, within E = e (|q'|^2 + |c'|^2) of the exact real
// squared distance.  Per query row, over the candidates whose order key is
// above the query's, each thread keeps the smallest upper bound acc + E (and
// its candidate) and the two smallest lower bounds acc - E (with the
// candidate of the smallest); E is taken per 32 columns at their largest
// candidate norm.  A query is settled when one candidate's upper bound U is
// below every other candidate's lower bound by a relative 2^-20 (so it is the
// unique nearest higher point in binary64 too) and band(U) is below the far
// bound of the block; lambda is that candidate and delta the square root of
// its canonical binary64 distance.  Every other query goes to the far phase
// with band(U) as its bound.

struct TcNearSmem {
  float a[2][kTcM * kTcK];
  float b[2][kTcN * kTcK];
  unsigned long long key[kTcN];  // order key per column (0: padding)
  float cmax[kTcN / 32];
  // the second column half's per-row results, merged by the first half
  float ub[kTcM], l1[kTcM], l2[kTcM];
  uint32_t ib[kTcM], il[kTcM];
  RunTable rt;
  unsigned long long mbar;
  uint32_t tmem;
  int nr;
  uint32_t item;
};

__device__ __forceinline__ float tc_band(float s, float mul, float add) {
  return __fadd_ru(__fmul_ru(s, mul), add);
}

// Coordinates of point `o` of an instance in the caller's input.
__device__ __forceinline__ Pt<8> tc_caller_pt(const void* __restrict__ pts, int dtype, uint64_t coord,
                                              int d, uint32_t o) {
  Pt<8> p;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    float v = 0.f;
    if (a < d) {
      const size_t e = coord + (size_t)o * d + a;
      v = dtype == 0 ? (float)__ldg((const int32_t*)pts + e) : __ldg((const float*)pts + e);
    }
    p.x[a] = v;
  }
  return p;
}

// The running bounds of one query (one column half): best upper bound ub and
// its candidate ib; the two smallest lower bounds l1 (candidate il) and l2.
struct NearBounds {
  float ub, l1, l2;
  uint32_t ib, il;
  __device__ __forceinline__ void init() {
    ub = l1 = l2 = INFINITY;
    ib = il = 0xffffffffu;
  }
  __device__ __forceinline__ void add_lower(float l, uint32_t id) {
    if (l < l1) {
      l2 = l1;
      l1 = l;
      il = id;
    } else if (l < l2) {
      l2 = l;
    }
  }
  __device__ __forceinline__ void add(float u, uint32_t idu, float l, float lo_rest) {
    if (u < ub) {
      ub = u;
      ib = idu;
    }
    add_lower(l, idu);
    add_lower(lo_rest, 0xfffffffeu);  // some other candidate of the same columns
  }
  __device__ __forceinline__ void merge(const NearBounds& o) {
    if (o.ub < ub) {
      ub = o.ub;
      ib = o.ib;
    }
    add_lower(o.l1, o.il);
    add_lower(o.l2, 0xfffffffeu);
  }
};

template <int G>
__global__ void __launch_bounds__(kTcThreads)
k_dep_near_tc(const float* __restrict__ spts, const unsigned long long* __restrict__ skey,
              ClassView cv, int32_t rho_skip, const void* __restrict__ pts, int dtype,
              const CutGeom* __restrict__ cuts, HashInfo* hi,
              const unsigned long long* __restrict__ hkeys, const uint2* __restrict__ hvals,
              const uint2* __restrict__ pieces, int32_t* __restrict__ lambda,
              double* __restrict__ delta, FarQueue fq, Counters* ctr, uint32_t poll_limit) {
  constexpr int DP = 8;
  extern __shared__ __align__(128) unsigned char tcn_smem_raw[];
  TcNearSmem& sm = *reinterpret_cast<TcNearSmem*>(tcn_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t npieces = hi->npieces;
  const uint32_t n = cv.N;
  const uint32_t mbar = smem_addr(&sm.mbar);
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&sm.tmem)), "r"(kTcN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;
  const int qrow = (warp & 3) * 32 + lane;
  const int chalf = warp >> 2;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(chalf * (kTcN / 2));
  uint32_t phase = 0;
  bool stop = false;

  while (!stop) {
    if (tid == 0) sm.item = atomicAdd(&hi->work, 1u);
    __syncthreads();
    const uint32_t item = sm.item;
    __syncthreads();
    if (item >= npieces) break;
    const uint2 pc = pieces[item];
    const uint32_t slot = pc.x & hmask;
    const unsigned long long hkey = hkeys[slot];
    const uint2 run = clip_run(hvals[slot], n);
    uint32_t inst = key_inst(hkey, S, ib);
    if (inst >= cv.ninst) inst = 0;
    const unsigned long long code = key_code(hkey, S, ib);
    const CutGeom& C = cuts[inst];
    const InstDev I = cv.instance(inst);
    const int R = C.R;
    const int cmax = (1 << (cv.geom[inst].B - C.k)) - 1;
    const float bmul = C.band_mul, badd = C.band_add, far32 = C.far32;
    const int32_t skip_below = max(rho_skip, C.skip);
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    uint32_t c0[G];
    unmorton<G>(code, c0);
    if (warp == 0) {
      Union<G> u;
      block_union<G>(c0, R, cmax, u);
      const int nrr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, sm.rt);
      if (lane == 0) sm.nr = nrr;
    }
    __syncthreads();
    const int nr = sm.nr;
    const uint32_t total = sm.rt.pre[nr];
    const uint32_t q0 = pc.y < run.x ? run.x : pc.y;
    const uint32_t qp = q0 + (uint32_t)qrow;
    const bool inq = qp < run.y;
    const Pt<DP> o = load_pt<DP>(spts, q0);
    Pt<DP> me;
#pragma unroll
    for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
    unsigned long long K = ~0ull;
    if (inq) {
      me = load_pt<DP>(spts, qp);
      K = skey[qp];
    }
    const bool act = inq && (int32_t)(K >> 32) >= skip_below;
    const unsigned long long Kc = act ? K : ~0ull;  // no candidate is above ~0
    float nq = 0.f;
    {
      float row[kTcK];
#pragma unroll
      for (int a = 0; a < DP; ++a) {
        const float t = inq ? me.x[a] - o.x[a] : 0.f;
        row[a] = t;
        nq = fmaf(t, t, nq);
      }
      row[8] = nq;
      row[9] = 1.f;
#pragma unroll
      for (int a = 10; a < kTcK; ++a) row[a] = 0.f;
      if (chalf == 0) put_row<kTcM>(sm.a, qrow, row);
    }
    NearBounds nb;
    nb.init();
    auto fetch = [&](uint32_t w, unsigned long long& kc) {
      Pt<DP> x;
#pragma unroll
      for (int a = 0; a < DP; ++a) x.x[a] = 0.f;
      kc = 0ull;
      const uint32_t e = w + (uint32_t)tid;
      if (e < total) {
        int lo = 0, hi2 = nr - 1;
        while (lo < hi2) {
          const int mid = (lo + hi2 + 1) >> 1;
          if (sm.rt.pre[mid] <= e) lo = mid;
          else hi2 = mid - 1;
        }
        const uint32_t src = sm.rt.start[lo] + (e - sm.rt.pre[lo]);
        x = load_pt<DP>(spts, src);
        kc = skey[src];
      }
      return x;
    };
    unsigned long long knext;
    Pt<DP> xnext = fetch(0, knext);
    for (uint32_t w0 = 0; w0 < total && !stop; w0 += kTcN) {
      {
        const int r = tid;
        float row[kTcK];
        float ncr = 0.f;
        if (w0 + (uint32_t)r < total) {
          float nc = 0.f;
#pragma unroll
          for (int a = 0; a < DP; ++a) {
            const float t = xnext.x[a] - o.x[a];
            row[a] = -2.f * t;
            nc = fmaf(t, t, nc);
          }
          row[8] = 1.f;
          row[9] = nc;
          ncr = nc;
          sm.key[r] = knext;
        } else {
#pragma unroll
          for (int a = 0; a < DP; ++a) row[a] = 0.f;
          row[8] = 0.f;
          row[9] = kTcFar;
          sm.key[r] = 0ull;
        }
        float m = ncr;
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
        if (lane == 0) sm.cmax[warp] = m;
#pragma unroll
        for (int a = 10; a < kTcK; ++a) row[a] = 0.f;
        put_row<kTcN>(sm.b, r, row);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t ab = smem_addr(sm.a[0]), al = smem_addr(sm.a[1]);
        const uint32_t bb = smem_addr(sm.b[0]), bl = smem_addr(sm.b[1]);
        const uint32_t as[3] = {ab, ab, al}, bs[3] = {bb, bl, bb};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
          for (int sp = 0; sp < 3; ++sp) {
            const uint64_t ad = smem_desc(as[sp] + ks * (kTcM * 32));
            const uint64_t bd = smem_desc(bs[sp] + ks * (kTcN * 32));
            const uint32_t accum = (ks | sp) ? 1u : 0u;
            asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n"
                         :: "r"(tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum) : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mbar) : "memory");
      }
      if (w0 + kTcN < total) xnext = fetch(w0 + kTcN, knext);
      const bool ok = mbar_wait(mbar, phase, poll_limit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {  // the MMA did not finish in time: record and stop
        if (tid == 0) set_status(cv.cls->status, kStatusTimeout);
        mbar_wait(mbar, phase ^ 1u, kTcWaitLimit);  // the MMA in flight, before TMEM is freed
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ncol = (int)min((uint32_t)kTcN, total - w0);
      for (int cl = 0; cl < kTcN / 2; cl += 32) {
        const int cb = chalf * (kTcN / 2) + cl;
        if (cb >= ncol) break;  // warp-uniform
        float v[32];
        tmem_ld32(trow + (uint32_t)cl, v);
        if (act) {
          // the two smallest accumulators among the higher candidates of
          // these 32 columns, and the candidate at the smallest
          float a1 = INFINITY, a2 = INFINITY;
          uint32_t i1 = 0xffffffffu;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const unsigned long long kc = sm.key[cb + j];
            const float x = kc > Kc ? v[j] : INFINITY;
            a2 = fminf(a2, fmaxf(a1, x));
            i1 = x < a1 ? key_id(kc) : i1;
            a1 = fminf(a1, x);
          }
          if (i1 != 0xffffffffu) {
            const float E = __fmul_ru(kTcErr, __fadd_ru(nq, sm.cmax[cb >> 5]));
            nb.add(__fadd_ru(a1, E), i1, __fsub_rd(a1, E), __fsub_rd(a2, E));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    // the two column halves of each query, then settle it or queue it
    if (chalf == 1) {
      sm.ub[qrow] = nb.ub;
      sm.l1[qrow] = nb.l1;
      sm.l2[qrow] = nb.l2;
      sm.ib[qrow] = nb.ib;
      sm.il[qrow] = nb.il;
    }
    __syncthreads();
    bool push = false;
    float s_hand = INFINITY;
    if (chalf == 0 && inq && !stop) {
      NearBounds other;
      other.ub = sm.ub[qrow];
      other.l1 = sm.l1[qrow];
      other.l2 = sm.l2[qrow];
      other.ib = sm.ib[qrow];
      other.il = sm.il[qrow];
      nb.merge(other);
      const uint32_t id = key_id(K);
      if (!act) {
        lambda[id] = -1;
        delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: skipped
      } else {
        bool settled = false;
        if (nb.ib != 0xffffffffu) {
          const float rest = nb.il == nb.ib ? nb.l2 : nb.l1;
          settled = tc_band(nb.ub, bmul, badd) < far32 && rest > __fmul_ru(nb.ub, 1.f + 0x1p-20f);
          s_hand = tc_band(nb.ub, bmul, badd);
        }
        if (settled) {
          const uint32_t ol = nb.ib - (uint32_t)I.out;
          lambda[id] = (int32_t)ol;
          delta[id] = sqrt(dist64<DP>(me, tc_caller_pt(pts, dtype, I.coord, I.d, ol)));
        } else {
          push = true;
        }
      }
    }
    const unsigned pm = __ballot_sync(kFull, push);
    uint32_t base = 0;
    if (lane == 0 && pm) base = atomicAdd(&ctr->queue_n, (unsigned)__popc(pm));
    base = __shfl_sync(kFull, base, 0);
    if (push) {
      const uint32_t slot2 = base + __popc(pm & lanemask_lt);
      fq.pos[slot2] = qp;
      fq.s1[slot2] = s_hand;
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcN) : "memory");
}

constexpr size_t kTcNearSmemBytes =
    sizeof(TcNearSmem) > 100 * 1024 ? sizeof(TcNearSmem) : 100 * 1024;
static_assert(sizeof(TcNearSmem) <= 200 * 1024, "shared-memory layout too large");

}  // namespace

void launch_density_tc(int g, const float* spts, const uint32_t* sid, const ClassView& cv,
                       const CutGeom* cuts, HashInfo* hi, const unsigned long long* hkeys,
                       const uint2* hvals, uint2* pieces, int32_t* rho_out,
                       unsigned long long* skey, Counters* ctr, cudaStream_t st) {
  if (cv.N == 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_density_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTcSmemBytes);
    cudaFuncSetAttribute(k_density_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTcSmemBytes);
    attr = true;
  }
  cudaMemsetAsync(&hi->work, 0, sizeof(uint32_t), st);
  cudaMemsetAsync(&hi->npieces, 0, sizeof(uint32_t), st);
  k_tc_pieces<<<sm_count() * 8u, 256, 0, st>>>(hi, hkeys, hvals, cv.N, pieces, sid, rho_out, skey,
                                                true, nullptr);
  const unsigned grid = sm_count() * 2u;  // two resident CTAs per SM take the pieces one by one
  const uint32_t poll = wait_limit(kTcWaitLimit);
  if (g == 3)
    k_density_tc<3><<<grid, kTcThreads, kTcSmemBytes, st>>>(spts, sid, cv, cuts, hi, hkeys, hvals,
                                                            pieces, rho_out, skey, ctr, poll);
  else
    k_density_tc<4><<<grid, kTcThreads, kTcSmemBytes, st>>>(spts, sid, cv, cuts, hi, hkeys, hvals,
                                                            pieces, rho_out, skey, ctr, poll);
  count_launches(2);
}


void launch_dep_near_tc(int g, const float* spts, const uint32_t* sid,
                        const unsigned long long* skey, const ClassView& cv, int32_t rho_skip,
                        const void* pts, int dtype, const CutGeom* cuts, HashInfo* hi,
                        const unsigned long long* hkeys, const uint2* hvals, uint2* pieces,
                        int32_t* lambda, double* delta, FarQueue q, Counters* ctr,
                        cudaStream_t st) {
  if (cv.N == 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dep_near_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTcNearSmemBytes);
    cudaFuncSetAttribute(k_dep_near_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTcNearSmemBytes);
    attr = true;
  }
  cudaMemsetAsync(&ctr->queue_n, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(&ctr->queue2_n, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(&hi->work, 0, sizeof(uint32_t), st);
  cudaMemsetAsync(&hi->npieces, 0, sizeof(uint32_t), st);
  k_tc_pieces<<<sm_count() * 8u, 256, 0, st>>>(hi, hkeys, hvals, cv.N, pieces, sid, nullptr,
                                                nullptr, false, lambda);
  const unsigned grid = sm_count() * 2u;
  const uint32_t poll = wait_limit(kTcWaitLimit);
  if (g == 3)
    k_dep_near_tc<3><<<grid, kTcThreads, kTcNearSmemBytes, st>>>(spts, skey, cv, rho_skip, pts, dtype,
                                                                 cuts, hi, hkeys, hvals, pieces,
                                                                 lambda, delta, q, ctr, poll);
  else
    k_dep_near_tc<4><<<grid, kTcThreads, kTcNearSmemBytes, st>>>(spts, skey, cv, rho_skip, pts, dtype,
                                                                 cuts, hi, hkeys, hvals, pieces,
                                                                 lambda, delta, q, ctr, poll);
  count_launches(2);
}

}  // namespace dpc
