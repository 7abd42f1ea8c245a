// density.cu -- rho_i = |{j : D(x_i, x_j) <= d_cut}| (Definition 1).
//
// One query per lane, 32 consecutive Morton-sorted queries per warp; the warp
// stages the union of its queries' grid blocks in shared memory (block.cuh)
// and each lane counts the points of its own (2R+1)^g block, reading every
// candidate as a broadcast.
//   FP32_CERT: s32 <= t_in counts, s32 > t_out does not.  Pairs in between
//              (about 1e-6 of d_cut^2 wide) are counted with the canonical
//              binary64 distance in a separate pass, taken only by a warp that
//              met one, so the hot loop stays float32.
//   FP64:      every pair is evaluated in binary64.
// Both give exactly the binary64 count.  The kernel also writes the order key
// of every sorted point, (rho << 32) | ~id.
#include <type_traits>

#include "block.cuh"
#include "internal.h"

namespace dpc {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

template <int DP>
constexpr int density_cap() { return DP == 8 ? 256 : 512; }

// Exact count of this lane's band pairs among the window's candidates (rare
// path, taken only by a warp that met a band pair in this window).
template <int DP, int G>
__device__ __noinline__ int2 band_recount(const RunTable& rt, int nr, const Union<G> u,
                                          uint32_t w0, uint32_t w1, const float* wpts,
                                          const uint32_t* c0, bool act, int R, Pt<DP> me,
                                          float t_in, float t_out, double dc2) {
  int in = 0, seen = 0;
  for_window_runs<G>(rt, nr, u, w0, w1, [&](uint32_t i0, uint32_t i1, const uint32_t* cc) {
    if (!(act && in_block<G>(c0, cc, R))) return;
    for (uint32_t i = i0; i < i1; ++i) {
      const Pt<DP> x = window_pt<DP>(wpts, i);
      const float s32 = dist32<DP>(me, x);
      if (s32 > t_in && s32 <= t_out) {
        ++seen;
        in += dist64<DP>(me, x) <= dc2;
      }
    }
  });
  return make_int2(in, seen);
}

// Resident blocks per SM the register budget must allow (shared memory
// allows 10 of the 2-D and 5 of the wider blocks).
template <int DP>
constexpr int density_min_blocks() { return DP == 2 ? 7 : 5; }

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads, density_min_blocks<DP>())
k_density(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
          const uint32_t* __restrict__ sid, ClassView cv, const CutGeom* __restrict__ cuts,
          const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
          const uint2* __restrict__ hvals, int32_t* __restrict__ rho_out,
          unsigned long long* __restrict__ skey, Counters* ctr) {
  constexpr int ND = real_dims<DP, G>();
  constexpr int kCap = density_cap<DP>();
  __shared__ __align__(16) float s_pts[kWarps * kCap * DP];
  __shared__ RunTable s_rt[kWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* wpts = s_pts + wib * kCap * DP;
  RunTable& rt = s_rt[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;

  unsigned long long band = 0, pairs = 0;
  for (uint32_t ch = blockIdx.x * kWarps + wib; ch < cv.nchunk; ch += gridDim.x * kWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const CutGeom& C = cuts[inst];
    const int k = C.k;
    const int R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const double dc2 = C.dc2;
    const float t_in = C.t_in, t_out = C.t_out;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    Pt<DP> me;
#pragma unroll
    for (int a = 0; a < DP; ++a) me.x[a] = 0.f;
    if (valid) me = load_pt<DP>(spts, p);
    const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
    uint32_t c0[G];
    unmorton<G>(valid ? mycell : 0ull, c0);
    const int nvalid = (int)min(32u, end - p0);
    int32_t count = 0;
    for_groups<G>(mycell, c0, valid, valid, nvalid, R, cmax, lane, [&](bool act, const Union<G>& u) {
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      const uint32_t total = rt.pre[nr];
      for (uint32_t w0 = 0; w0 < total; w0 += kCap) {
        const uint32_t w1 = min(total, w0 + (uint32_t)kCap);
        __syncwarp();
        stage_runs<DP, false>(rt, nr, w0, w1, spts, nullptr, wpts, nullptr, lane);
        __syncwarp();
        int32_t c = 0, c2 = 0;
        for_window_runs<G>(rt, nr, u, w0, w1, [&](uint32_t i0, uint32_t i1, const uint32_t* cc) {
          const bool need = act && in_block<G>(c0, cc, R);
          if (!__any_sync(kFull, need)) return;
          if (need) pairs += i1 - i0;
          // a lane outside this cell's block compares against -1: never counts
          const float ti = need ? t_in : -1.f, to = need ? t_out : -1.f;
          const double dl = need ? dc2 : -1.0;
#pragma unroll 4
          for (uint32_t i = i0; i < i1; ++i) {
            const Pt<DP> x = window_pt<DP>(wpts, i);
            if constexpr (F64) {
              c += dist64<DP, ND>(me, x) <= dl;
            } else {
              const float s32 = dist32<DP, ND>(me, x);
              c += s32 <= ti;
              c2 += s32 <= to;
            }
          }
        });
        if constexpr (!F64) {
          if (__any_sync(kFull, c2 != c)) {
            const int2 r = band_recount<DP, G>(rt, nr, u, w0, w1, wpts, c0, act && c2 != c, R, me,
                                               t_in, t_out, dc2);
            c += r.x;
            band += r.y;
          }
        }
        count += c;
      }
      __syncwarp();
    });
    if (valid) {
      const uint32_t id = sid[p];
      rho_out[id] = count;
      skey[p] = order_key(count, id);
    }
  }
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
  if (lane == 0 && pairs) atomicAdd(&ctr->pairs, pairs);
  if constexpr (!F64) {
    for (int o = 16; o > 0; o >>= 1) band += __shfl_xor_sync(kFull, band, o);
    if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

// ---------------------------------------------------------------------------
// Segment form: the 32 points of a chunk are split into segments of equal
// level-k cell; for each segment the warp looks up that cell's (2R+1)^g block
// and spreads the block's candidates over the lanes (V per lane, held in
// registers), then walks the segment's queries one by one: every lane
// compares its V candidates with the query (read as a broadcast) and one warp
// reduction gives the query's count.  No lane evaluates a candidate outside
// the query's block, so the work is exactly the block's pairs.
// In float32 the lane holds its candidates negated, two per packed register,
// and evaluates dist32 for both at once (packed add / mul / fma: the same
// rounding as the scalar sequence, so the certified band is unchanged); a
// pair counts when s - up(t_in) is negative (its sign bit), and one unsigned
// minimum per lane over the bit patterns of s finds band pairs, which are
// recounted in binary64 after the window.  Small V (4 slots in 3-D) keeps the
// kernel at 80 registers, 6 blocks per SM: the loop is latency-bound, and more
// resident warps pay more than longer windows.

// Exact count of the band pairs of queries qa and qb (sorted positions) among
// this lane's candidates of window w0 (rare path: a warp takes it only for the
// query pairs of a window that met a band pair, after the window's passes).
// The candidates are loaded again one slot at a time, so neither the hot loop
// nor this pass holds a window's copy.  Returns (binary64 counts of a | b << 16,
// band pairs seen of a | b << 16), summed over the warp.
template <int DP, int V, int ND>
__device__ __forceinline__ uint2 seg_band_recount(const RunTable& rt, int nr, uint32_t w0,
                                                  uint32_t total, const float* __restrict__ spts,
                                                  int lane, uint32_t qa, uint32_t qb, float t_in,
                                                  float t_out, double dc2) {
  const Pt<DP> xa = load_pt<DP>(spts, qa);
  const Pt<DP> xb = load_pt<DP>(spts, qb);
  unsigned in = 0, seen = 0;
#pragma unroll 1
  for (uint32_t e = w0 + lane; e < total && e < w0 + 32u * V; e += 32u) {
    int lo = 0, hi = nr - 1;  // the run holding candidate e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rt.pre[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const Pt<DP> x = load_pt<DP>(spts, rt.start[lo] + (e - rt.pre[lo]));
    const float sa = dist32<DP, ND>(xa, x);
    const float sb = dist32<DP, ND>(xb, x);
    if (sa > t_in && sa <= t_out) {
      ++seen;
      in += dist64<DP, ND>(xa, x) <= dc2 ? 1u : 0u;
    }
    if (sb > t_in && sb <= t_out) {
      seen += 0x10000u;
      in += dist64<DP, ND>(xb, x) <= dc2 ? 0x10000u : 0u;
    }
  }
  return make_uint2(__reduce_add_sync(kFull, in), __reduce_add_sync(kFull, seen));
}

template <int DP>
constexpr int seg_v() { return DP == 2 ? 8 : (DP == 4 ? 4 : 2); }

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads, (F64 || G >= 4) ? 5 : 6)
k_density_seg(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
              const uint32_t* __restrict__ sid, ClassView cv, const CutGeom* __restrict__ cuts,
              const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
              const uint2* __restrict__ hvals, int32_t* __restrict__ rho_out,
              unsigned long long* __restrict__ skey, Counters* ctr, int seg_cells) {
  constexpr int ND = real_dims<DP, G>();
  constexpr int V = seg_v<DP>();
  constexpr uint32_t W = 32u * V;
  __shared__ RunTable s_rt[kWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  RunTable& rt = s_rt[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;

  unsigned long long band = 0, pairs = 0;
  for (uint32_t ch = blockIdx.x * kWarps + wib; ch < cv.nchunk; ch += gridDim.x * kWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const CutGeom& C = cuts[inst];
    const int k = C.k;
    const int R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const double dc2 = C.dc2;
    const float t_in = C.t_in, t_out = C.t_out;
    const BandBits bb = band_bits(t_in, t_out);
    // s <= t_in  <=>  s - up(t_in) < 0, with up(t_in) the next float above
    const f32x2 ntin2 = pack2(-next_up(t_in), -next_up(t_in));
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
    const int nvalid = (int)min(32u, end - p0);
    int32_t acc = 0;  // lane j: the count of query p0 + j
    int s = 0;
    while (s < nvalid) {
      Union<G> u;
      const int e = super_segment<G>(mycell, valid, s, nvalid, R, cmax, seg_cells, lane, u);  // queries s .. e-1
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      const uint32_t total = rt.pre[nr];
      pairs += (unsigned long long)(e - s) * total;
      for (uint32_t w0 = 0; w0 < total; w0 += W) {
        Pt<DP> cand[V];
        load_window<DP, V>(rt, nr, w0, total, spts, lane, cand);
        // slots of this window that hold candidates (warp-uniform)
        const int vn = (int)min((uint32_t)V, (total - w0 + 31u) / 32u);
        if constexpr (F64) {
          for (int j = s; j < e; j += 2) {
            const bool two = j + 1 < e;
            const Pt<DP> xa = load_pt<DP>(spts, p0 + j);
            const Pt<DP> xb = load_pt<DP>(spts, p0 + (two ? j + 1 : j));
            unsigned c = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if (v >= vn) break;
              c += (dist64<DP, ND>(xa, cand[v]) <= dc2) ? 1u : 0u;
              c += (dist64<DP, ND>(xb, cand[v]) <= dc2) ? 0x10000u : 0u;
            }
            c = __reduce_add_sync(kFull, c);
            if (lane == j) acc += (int32_t)(c & 0xffffu);
            if (two && lane == j + 1) acc += (int32_t)(c >> 16);
          }
        } else {
          // the lane's candidates negated, two slots per packed register; a
          // slot past the window's end holds +inf (distance +inf: never
          // counted, never in the band)
          f32x2 nc[V / 2][ND];
#pragma unroll
          for (int i = 0; i < V / 2; ++i) {
            const bool ok0 = w0 + (uint32_t)lane + 64u * i < total;
            const bool ok1 = w0 + (uint32_t)lane + 64u * i + 32u < total;
#pragma unroll
            for (int k = 0; k < ND; ++k)
              nc[i][k] = pack2(ok0 ? -cand[2 * i].x[k] : INFINITY, ok1 ? -cand[2 * i + 1].x[k] : INFINITY);
          }
          // two queries per pass over the lane's candidate pairs (independent
          // chains); their per-lane counts (at most V each) share one 32-bit
          // word per reduction, and one unsigned minimum per lane tells
          // whether any of its pairs fell in the band
          uint32_t bandq = 0;  // bit j: queries j and j + 1 met a band pair
          auto passes = [&](auto full_window) {
            constexpr bool kFullWindow = decltype(full_window)::value;
            const int vp = (vn + 1) >> 1;
            for (int j = s; j < e; j += 2) {
              const bool two = j + 1 < e;
              const Pt<DP> xa = load_pt<DP>(spts, p0 + j);
              const Pt<DP> xb = load_pt<DP>(spts, p0 + (two ? j + 1 : j));
              f32x2 qa[ND], qb[ND];
#pragma unroll
              for (int k = 0; k < ND; ++k) {
                qa[k] = pack2(xa.x[k], xa.x[k]);
                qb[k] = pack2(xb.x[k], xb.x[k]);
              }
              uint32_t na = 0, nb = 0, mband = 0xffffffffu;
#pragma unroll
              for (int i = 0; i < V / 2; ++i) {
                if (!kFullWindow && i >= vp) break;
                const f32x2 sa = dist32x2<ND>(qa, nc[i]);
                const f32x2 sb = dist32x2<ND>(qb, nc[i]);
                na += sign_count2(add2(sa, ntin2));
                nb += sign_count2(add2(sb, ntin2));
                mband = min(mband, band_min2(sa, bb.lo));
                mband = min(mband, band_min2(sb, bb.lo));
              }
              unsigned c = na + (nb << 16);
              c = __reduce_add_sync(kFull, c);
              // band pairs: recounted in binary64 after the window's passes
              if (__any_sync(kFull, mband < bb.width)) bandq |= 1u << j;
              if (lane == j) acc += (int32_t)(c & 0xffffu);
              if (two && lane == j + 1) acc += (int32_t)(c >> 16);
            }
          };
          if (vn == V) passes(std::true_type{});
          else passes(std::false_type{});
          while (bandq) {
            const int j = __ffs(bandq) - 1;
            bandq &= bandq - 1u;
            const bool two = j + 1 < e;
            const uint2 r = seg_band_recount<DP, V, ND>(rt, nr, w0, total, spts, lane, p0 + j,
                                                        p0 + (two ? j + 1 : j), t_in, t_out, dc2);
            if (lane == j) acc += (int32_t)(r.x & 0xffffu);
            if (two && lane == j + 1) acc += (int32_t)(r.x >> 16);
            if (lane == 0) band += (r.y & 0xffffu) + (two ? (r.y >> 16) : 0u);
          }
        }
      }
      s = e;
    }
    if (valid) {
      const uint32_t id = sid[p];
      rho_out[id] = acc;
      skey[p] = order_key(acc, id);
    }
  }
  if (lane == 0 && pairs) atomicAdd(&ctr->pairs, pairs);
  if constexpr (!F64) {
    if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

// candidate slots per lane of the pair layout (its per-slot counts need
// registers of their own)
template <int DP>
constexpr int pairs_v() { return DP == 2 ? 8 : (DP == 4 ? 8 : 4); }

// Pair layout (symmetric): every unordered pair within d_cut is evaluated
// once and counted for both points.  The work layout is k_density_seg's
// (segments of equal cell, the block's candidates spread over the lanes, two
// queries per pass), but a segment in cell A only takes the cells B of its
// block that follow A in Morton order, plus the points of A itself that
// follow the query in sorted order.  A query's count stays in a register and
// each candidate's in a register per slot; both go to a position-indexed
// counter with one atomic add per window (candidates) or per chunk (queries).
// cnt2 is the low 32-bit word of each sorted point's 64-bit order key slot
// (index 2p), zeroed before; k_pairs_finish turns it into rho and the key.
template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kThreads, DP == 2 ? 5 : 4)
k_density_pairs(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
                ClassView cv, const CutGeom* __restrict__ cuts, const HashInfo* __restrict__ hi,
                const unsigned long long* __restrict__ hkeys, const uint2* __restrict__ hvals,
                uint32_t* __restrict__ cnt2, Counters* ctr) {
  constexpr int ND = real_dims<DP, G>();
  constexpr int V = pairs_v<DP>();
  constexpr uint32_t W = 32u * V;
  __shared__ RunTable s_rt[kWarps];
  __shared__ RunTable s_rt2[kWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  RunTable& rt = s_rt[wib];
  RunTable& rt2 = s_rt2[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;

  unsigned long long band = 0, pairs = 0;
  for (uint32_t ch = blockIdx.x * kWarps + wib; ch < cv.nchunk; ch += gridDim.x * kWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const CutGeom& C = cuts[inst];
    const int k = C.k;
    const int R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const double dc2 = C.dc2;
    const float t_in = C.t_in, t_out = C.t_out;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;
    const uint32_t p = p0 + lane;
    const bool valid = p < end;
    const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
    const int nvalid = (int)min(32u, end - p0);
    int32_t acc = valid ? 1 : 0;  // lane j: query p0 + j (itself, then its pairs)
    int s = 0;
    while (s < nvalid) {
      const unsigned long long cell = __shfl_sync(kFull, mycell, s);
      const int e = s + __popc(__ballot_sync(kFull, valid && mycell == cell));  // queries s .. e-1
      uint32_t c0[G];
      unmorton<G>(cell, c0);
      Union<G> u;
      block_union<G>(c0, R, cmax, u);
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      // OWN = false: the cells after A; OWN = true: A's points after the
      // segment's first query (a pair counts only if the candidate follows
      // the query)
      auto scan = [&](const RunTable& tab, int ntab, auto own_tag) {
        constexpr bool OWN = decltype(own_tag)::value;
        const uint32_t total = tab.pre[ntab];
        pairs += (unsigned long long)(e - s) * total;
        for (uint32_t w0 = 0; w0 < total; w0 += W) {
          Pt<DP> cand[V];
          load_window<DP, V>(tab, ntab, w0, total, spts, lane, cand);
          const int vn = (int)min((uint32_t)V, (total - w0 + 31u) / 32u);
          // OWN: one run, so slot v of this lane holds position pbase + 32 v
          const uint32_t pbase = OWN ? tab.start[0] + w0 + lane : 0u;
          // this lane's candidates' counts, two 16-bit halves per word
          uint32_t cc[(V + 1) / 2];
#pragma unroll
          for (int v = 0; v < (V + 1) / 2; ++v) cc[v] = 0u;
          for (int j = s; j < e; j += 2) {
            const bool two = j + 1 < e;
            const uint32_t qa = p0 + j, qb = p0 + (two ? j + 1 : j);
            const Pt<DP> xa = load_pt<DP>(spts, qa);
            const Pt<DP> xb = load_pt<DP>(spts, qb);
            int32_t cnt_a, cnt_b;
            if constexpr (F64) {
              unsigned c = 0;
#pragma unroll
              for (int v = 0; v < V; ++v) {
                if (v >= vn) break;
                const uint32_t pv = pbase + 32u * v;
                const bool ea = (!OWN || pv > qa) && dist64<DP, ND>(xa, cand[v]) <= dc2;
                const bool eb = two && (!OWN || pv > qb) && dist64<DP, ND>(xb, cand[v]) <= dc2;
                c += (ea ? 1u : 0u) + (eb ? 0x10000u : 0u);
                cc[v >> 1] += ((ea ? 1u : 0u) + (eb ? 1u : 0u)) << (16 * (v & 1));
              }
              c = __reduce_add_sync(kFull, c);
              cnt_a = (int32_t)(c & 0xffffu);
              cnt_b = (int32_t)(c >> 16);
            } else {
              unsigned ci = 0, co = 0;
#pragma unroll
              for (int v = 0; v < V; ++v) {
                if (v >= vn) break;
                const uint32_t pv = pbase + 32u * v;
                const float sa0 = dist32<DP, ND>(xa, cand[v]);
                const float sb0 = dist32<DP, ND>(xb, cand[v]);
                // a pair that does not count is moved past every threshold
                const float sa = (!OWN || pv > qa) ? sa0 : INFINITY;
                const float sb = (two && (!OWN || pv > qb)) ? sb0 : INFINITY;
                const bool ia = sa <= t_in, ib2 = sb <= t_in;
                ci += (ia ? 1u : 0u) + (ib2 ? 0x10000u : 0u);
                co += (sa <= t_out ? 1u : 0u) + (sb <= t_out ? 0x10000u : 0u);
                cc[v >> 1] += ((ia ? 1u : 0u) + (ib2 ? 1u : 0u)) << (16 * (v & 1));
              }
              ci = __reduce_add_sync(kFull, ci);
              co = __reduce_add_sync(kFull, co);
              cnt_a = (int32_t)(ci & 0xffffu);
              cnt_b = (int32_t)(ci >> 16);
              if (co != ci) {  // band pairs: recount them in binary64
                unsigned in = 0, seen = 0;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                  if (v >= vn) break;
                  const uint32_t pv = pbase + 32u * v;
                  const float sa = (!OWN || pv > qa) ? dist32<DP, ND>(xa, cand[v]) : INFINITY;
                  const float sb = (two && (!OWN || pv > qb)) ? dist32<DP, ND>(xb, cand[v]) : INFINITY;
                  if (sa > t_in && sa <= t_out) {
                    ++seen;
                    const bool x = dist64<DP, ND>(xa, cand[v]) <= dc2;
                    in += x ? 1u : 0u;
                    cc[v >> 1] += (x ? 1u : 0u) << (16 * (v & 1));
                  }
                  if (sb > t_in && sb <= t_out) {
                    seen += 0x10000u;
                    const bool x = dist64<DP, ND>(xb, cand[v]) <= dc2;
                    in += x ? 0x10000u : 0u;
                    cc[v >> 1] += (x ? 1u : 0u) << (16 * (v & 1));
                  }
                }
                in = __reduce_add_sync(kFull, in);
                seen = __reduce_add_sync(kFull, seen);
                cnt_a += (int32_t)(in & 0xffffu);
                cnt_b += (int32_t)(in >> 16);
                if (lane == 0) band += (seen & 0xffffu) + (seen >> 16);
              }
            }
            if (lane == j) acc += cnt_a;
            if (two && lane == j + 1) acc += cnt_b;
          }
          // the candidates' counts, at their positions (found again in the run table)
          {
            const uint32_t e0 = w0 + lane;
            int lo = 0, hi = ntab - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (tab.pre[mid] <= e0) lo = mid;
              else hi = mid - 1;
            }
            int r = lo;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const uint32_t c = (cc[v >> 1] >> (16 * (v & 1))) & 0xffffu;
              const uint32_t ev = e0 + 32u * v;
              if (ev >= total) break;
              while (r + 1 < ntab && tab.pre[r + 1] <= ev) ++r;
              if (c) atomicAdd(&cnt2[2 * (size_t)(tab.start[r] + (ev - tab.pre[r]))], c);
            }
          }
        }
      };
      // the block's cells after A (Morton order)
      const int nb = filter_runs<G>(rt, nr, u, rt2, lane, [&](const uint32_t* cc) {
        return morton<G>(cc) > cell;
      });
      scan(rt2, nb, std::false_type());
      // A itself: its points after the segment's first query
      {
        const uint2 run = clip_run(hash_find(hkeys, hvals, hmask, hb | cell), n);
        const uint32_t a0 = max(run.x, p0 + (uint32_t)s + 1u);
        __syncwarp();
        if (lane == 0) {
          rt2.pre[0] = 0u;
          rt2.start[0] = a0;
          rt2.cell[0] = 0u;
          rt2.pre[1] = run.y > a0 ? run.y - a0 : 0u;
        }
        __syncwarp();
        scan(rt2, 1, std::true_type());
      }
      s = e;
    }
    if (valid) atomicAdd(&cnt2[2 * (size_t)p], (uint32_t)acc);
  }
  if (lane == 0 && pairs) atomicAdd(&ctr->pairs, pairs);
  if constexpr (!F64) {
    if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

// Counts of the pair layout -> rho (by output id) and the order keys.
__global__ void k_pairs_finish(const uint32_t* __restrict__ sid, uint32_t n, int32_t* __restrict__ rho_out,
                               unsigned long long* __restrict__ skey) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t c = reinterpret_cast<const uint32_t*>(skey)[2 * (size_t)p];
    const uint32_t id = sid[p];
    rho_out[id] = (int32_t)c;
    skey[p] = order_key((int32_t)c, id);
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
void density_dg(bool fp64, int layout, const float* spts, const unsigned long long* scode,
                const uint32_t* sid, const ClassView& cv, const CutGeom* cuts, const HashInfo* hi,
                const unsigned long long* hkeys, const uint2* hvals, int32_t* rho_out,
                unsigned long long* skey, Counters* ctr, int seg_cells, cudaStream_t st) {
  const unsigned grid = grid_for(cv.nchunk, kWarps, sm_count() * 64u);
  if (layout == kLayoutPairs) {
    cudaMemsetAsync(skey, 0, sizeof(unsigned long long) * cv.N, st);
    uint32_t* cnt2 = reinterpret_cast<uint32_t*>(skey);
    if (fp64)
      k_density_pairs<DP, G, true><<<grid, kThreads, 0, st>>>(spts, scode, cv, cuts, hi, hkeys, hvals,
                                                              cnt2, ctr);
    else
      k_density_pairs<DP, G, false><<<grid, kThreads, 0, st>>>(spts, scode, cv, cuts, hi, hkeys, hvals,
                                                               cnt2, ctr);
    k_pairs_finish<<<grid_for(cv.N, 256, sm_count() * 16u), 256, 0, st>>>(sid, cv.N, rho_out, skey);
    count_launches(1);
  } else if (layout == kLayoutSegment) {
    if (fp64)
      k_density_seg<DP, G, true><<<grid, kThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys,
                                                            hvals, rho_out, skey, ctr, seg_cells);
    else
      k_density_seg<DP, G, false><<<grid, kThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys,
                                                             hvals, rho_out, skey, ctr, seg_cells);
  } else {
    if (fp64)
      k_density<DP, G, true><<<grid, kThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys, hvals,
                                                        rho_out, skey, ctr);
    else
      k_density<DP, G, false><<<grid, kThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys,
                                                         hvals, rho_out, skey, ctr);
  }
  count_launches(1);
}

}  // namespace

void launch_density(int dp, int g, bool fp64, int layout, const float* spts,
                    const unsigned long long* scode, const uint32_t* sid, const ClassView& cv,
                    const CutGeom* cuts, HashInfo* hi, const unsigned long long* hkeys,
                    const uint2* hvals, uint2* pieces, int32_t* rho_out,
                    unsigned long long* skey, Counters* ctr, cudaStream_t st, int seg_cells) {
  if (cv.N == 0) return;
  if (layout == kLayoutTensor) {
    if (dp == 8 && !fp64 && pieces) {
      launch_density_tc(g, spts, sid, cv, cuts, hi, hkeys, hvals, pieces, rho_out, skey, ctr, st);
      return;
    }
    layout = kLayoutSegment;
  }
  if (layout == kLayoutCell) {
    launch_density_cell(dp, g, fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr,
                        st);
    return;
  }
  if (g == 1) density_dg<2, 1>(fp64, layout, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, seg_cells, st);
  else if (g == 2) density_dg<2, 2>(fp64, layout, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, seg_cells, st);
  else if (g == 3) density_dg<4, 3>(fp64, layout, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, seg_cells, st);
  else if (dp == 4) density_dg<4, 4>(fp64, layout, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, seg_cells, st);
  else density_dg<8, 4>(fp64, layout, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, seg_cells, st);
}

void launch_keys_from_rho(const int32_t* rho, const uint32_t* sid, uint32_t n,
                          unsigned long long* skey, cudaStream_t st) {
  if (n == 0) return;
  k_keys_from_rho<<<grid_for(n, 256, sm_count() * 16u), 256, 0, st>>>(rho, sid, n, skey);
  count_launches(1);
}

}  // namespace dpc
