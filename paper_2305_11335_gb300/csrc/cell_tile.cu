// cell_tile.cu -- the density (Definition 1) and near-dependent
// (Definitions 2-3) kernels in the cell layout.
//
// Every query of one level-k grid cell needs exactly the same candidates: the
// points of the (2R+1)^g block of cells around it.  So the unit of work here
// is one occupied cell: a warp looks the block's cells up in the occupied-
// cell hash (one cell per lane), stages the block's points (and, for the
// dependent search, their order keys) in its slice of shared memory, and then
// every lane evaluates its queries against the staged candidates with
// broadcast reads.  A cell with m < 32 points gives each query L = 32 /
// 2^ceil(log2 m) lanes that split the candidates between them and combine
// their partial results with L - 1 shuffles at the end; a cell with 32 or more
// points gives each lane up to kQB queries, so every staged candidate read
// serves several of them.  No per-candidate search of the run table, no
// per-query warp reduction, no candidate outside the query's block.
//
// A warp owns the cells that start in its 32-point chunk of the sorted order
// (a cell whose run continues past the chunk is still the warp's); blocks
// larger than the shared-memory window are streamed window by window.
//
// Exactness is the same as in the other layouts: density counts s32 <= t_in
// and re-evaluates the pairs with t_in < s32 <= t_out in binary64; the near
// search keeps the two smallest s32 among the higher candidates and settles a
// query only when its winner is alone in its float32 error band and closer
// than anything outside the block can be; the rest go to the far phase.
#include "block.cuh"
#include "internal.h"

namespace dpc {
namespace {

constexpr int kCellWarps = 4;
constexpr int kCellThreads = kCellWarps * 32;
constexpr int kQB = 2;  // queries per lane (cells of 32 points or more)

// candidates staged per warp and window
template <int DP>
constexpr int cell_cap() { return DP == 2 ? 512 : (DP == 4 ? 256 : 128); }

__device__ __forceinline__ float band_of_cell(float s, float mul, float add) {
  return __fadd_ru(__fmul_ru(s, mul), add);
}

// Lanes per query for a cell of m points (m >= 1): 32 >> ceil(log2 m) below
// 32 points, else 1.
__device__ __forceinline__ int lanes_per_query(uint32_t m) {
  if (m >= 32) return 1;
  return 32 >> (32 - __clz((int)m - 1));
}

// The cells starting in this warp's chunk, one by one: fn(first, cell code)
// with the warp's run table filled with the cell's block.  Returns nothing;
// fn sees the block size as rt.pre[nr].
template <int G, typename Fn>
__device__ __forceinline__ void for_chunk_cells(const unsigned long long* __restrict__ scode,
                                                const InstDev& I, uint32_t p0, uint32_t end,
                                                int S, int ib, int shift, int lane, Fn fn) {
  const uint32_t p = p0 + lane;
  const bool valid = p < end;
  const unsigned long long mycell = valid ? (key_code(scode[p], S, ib) >> shift) : ~0ull;
  const unsigned long long prev =
      (valid && p > I.start) ? (key_code(scode[p - 1], S, ib) >> shift) : ~0ull - 1ull;
  unsigned starts = __ballot_sync(kFull, valid && mycell != prev);
  while (starts) {
    const int s = __ffs(starts) - 1;
    starts &= starts - 1u;
    fn(p0 + (uint32_t)s, __shfl_sync(kFull, mycell, s));
  }
}

// Length of the run that starts at `first` in the run table (the query cell
// is one of the block's runs).
__device__ __forceinline__ uint32_t own_run_length(const RunTable& rt, int nr, uint32_t first,
                                                   int lane) {
  uint32_t len = 0;
  for (int base = 0; base < nr; base += 32) {
    const int i = base + lane;
    const bool hit = i < nr && rt.start[i] == first;
    const unsigned m = __ballot_sync(kFull, hit);
    if (m) {
      const int w = base + __ffs(m) - 1;
      len = rt.pre[w + 1] - rt.pre[w];
      break;
    }
  }
  return len;
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kCellThreads)
k_density_cell(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
               const uint32_t* __restrict__ sid, ClassView cv, const CutGeom* __restrict__ cuts,
               const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
               const uint2* __restrict__ hvals, int32_t* __restrict__ rho_out,
               unsigned long long* __restrict__ skey, Counters* ctr) {
  constexpr int ND = real_dims<DP, G>();
  constexpr int CAP = cell_cap<DP>();
  __shared__ __align__(16) float s_pts[kCellWarps * CAP * DP];
  __shared__ RunTable s_rt[kCellWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* wpts = s_pts + wib * CAP * DP;
  RunTable& rt = s_rt[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;
  unsigned long long band = 0, pairs = 0;

  for (uint32_t ch = blockIdx.x * kCellWarps + wib; ch < cv.nchunk; ch += gridDim.x * kCellWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const InstDev I = cv.instance(inst);
    const CutGeom& C = cuts[inst];
    const int k = C.k, R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const double dc2 = C.dc2;
    const float t_in = C.t_in, t_out = C.t_out;
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;

    for_chunk_cells<G>(scode, I, p0, end, S, ib, shift, lane, [&](uint32_t first,
                                                                   unsigned long long cell) {
      uint32_t c0[G];
      unmorton<G>(cell, c0);
      Union<G> u;
      block_union<G>(c0, R, cmax, u);
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      const uint32_t T = rt.pre[nr];
      const uint32_t m = own_run_length(rt, nr, first, lane);
      pairs += (unsigned long long)m * T;
      for (uint32_t qbase = 0; qbase < m; qbase += 32u * kQB) {
        const uint32_t mq = min(m - qbase, 32u * kQB);
        const int L = lanes_per_query(mq);
        const int nqb = mq >= 32 ? (int)((mq + 31u) / 32u) : 1;
        const int sub = lane & (L - 1);
        uint32_t qi[kQB];
        bool has[kQB];
        Pt<DP> x[kQB];
        int32_t cnt[kQB];
#pragma unroll
        for (int b = 0; b < kQB; ++b) {
          qi[b] = qbase + (uint32_t)(b * 32 + lane / L);
          has[b] = b < nqb && qi[b] < m;
          x[b] = load_pt<DP>(spts, first + (has[b] ? qi[b] : 0u));
          cnt[b] = 0;
        }
        for (uint32_t w0 = 0; w0 < T; w0 += CAP) {
          const uint32_t w1 = min(T, w0 + (uint32_t)CAP);
          const int nw = (int)(w1 - w0);
          __syncwarp();
          stage_runs<DP, false>(rt, nr, w0, w1, spts, nullptr, wpts, nullptr, lane);
          __syncwarp();
          if constexpr (F64) {
#pragma unroll 4
            for (int c = sub; c < nw; c += L) {
              const Pt<DP> y = window_pt<DP>(wpts, (uint32_t)c);
#pragma unroll
              for (int b = 0; b < kQB; ++b)
                if (b < nqb) cnt[b] += dist64<DP, ND>(x[b], y) <= dc2 ? 1 : 0;
            }
          } else {
            int32_t ci[kQB], co[kQB];
#pragma unroll
            for (int b = 0; b < kQB; ++b) ci[b] = co[b] = 0;
#pragma unroll 4
            for (int c = sub; c < nw; c += L) {
              const Pt<DP> y = window_pt<DP>(wpts, (uint32_t)c);
#pragma unroll
              for (int b = 0; b < kQB; ++b) {
                if (b < nqb) {
                  const float s = dist32<DP, ND>(x[b], y);
                  ci[b] += s <= t_in ? 1 : 0;
                  co[b] += s <= t_out ? 1 : 0;
                }
              }
            }
#pragma unroll
            for (int b = 0; b < kQB; ++b) {
              if (b < nqb && co[b] != ci[b]) {  // band pairs of this window: binary64 decides
                for (int c = sub; c < nw; c += L) {
                  const Pt<DP> y = window_pt<DP>(wpts, (uint32_t)c);
                  const float s = dist32<DP, ND>(x[b], y);
                  if (s > t_in && s <= t_out) {
                    ++band;
                    ci[b] += dist64<DP, ND>(x[b], y) <= dc2 ? 1 : 0;
                  }
                }
              }
              cnt[b] += ci[b];
            }
          }
        }
#pragma unroll
        for (int b = 0; b < kQB; ++b) {
          if (b >= nqb) break;  // warp-uniform
          for (int o = L >> 1; o > 0; o >>= 1) cnt[b] += __shfl_xor_sync(kFull, cnt[b], o);
          if (has[b] && sub == 0) {
            const uint32_t pq = first + qi[b];
            const uint32_t id = sid[pq];
            rho_out[id] = cnt[b];
            skey[pq] = order_key(cnt[b], id);
          }
        }
      }
    });
  }
  for (int o = 16; o > 0; o >>= 1) {
    band += __shfl_xor_sync(kFull, band, o);
  }
  if (lane == 0 && pairs) atomicAdd(&ctr->pairs, pairs);
  if constexpr (!F64) {
    if (lane == 0 && band) atomicAdd(&ctr->band_pairs, band);
  }
}

// Coordinates of point `o` of an instance in the caller's input (the values
// the sorted float copy holds).
template <int DP>
__device__ __forceinline__ Pt<DP> caller_pt(const void* __restrict__ pts, int dtype, uint64_t coord,
                                            int d, uint32_t o) {
  Pt<DP> p;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
    float v = 0.f;
    if (a < d) {
      const size_t e = coord + (size_t)o * d + a;
      v = dtype == 0 ? (float)__ldg((const int32_t*)pts + e) : __ldg((const float*)pts + e);
    }
    p.x[a] = v;
  }
  return p;
}

template <int DP, int G, bool F64>
__global__ void __launch_bounds__(kCellThreads)
k_dep_near_cell(const float* __restrict__ spts, const unsigned long long* __restrict__ scode,
                const unsigned long long* __restrict__ skey, ClassView cv, int32_t rho_skip,
                const void* __restrict__ pts, int dtype, const CutGeom* __restrict__ cuts,
                const HashInfo* __restrict__ hi, const unsigned long long* __restrict__ hkeys,
                const uint2* __restrict__ hvals, int32_t* __restrict__ lambda,
                double* __restrict__ delta, FarQueue q, Counters* ctr) {
  constexpr int ND = real_dims<DP, G>();
  constexpr int CAP = cell_cap<DP>();
  __shared__ __align__(16) float s_pts[kCellWarps * CAP * DP];
  __shared__ unsigned long long s_key[kCellWarps * CAP];
  __shared__ RunTable s_rt[kCellWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* wpts = s_pts + wib * CAP * DP;
  unsigned long long* wkey = s_key + wib * CAP;
  RunTable& rt = s_rt[wib];
  const int S = cv.cls->S, ib = cv.cls->ib;
  const uint32_t hmask = hi->hmask;
  const uint32_t n = cv.N;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  for (uint32_t ch = blockIdx.x * kCellWarps + wib; ch < cv.nchunk; ch += gridDim.x * kCellWarps) {
    uint32_t inst, p0, end;
    cv.chunk(ch, inst, p0, end);
    const InstDev I = cv.instance(inst);
    const CutGeom& C = cuts[inst];
    const int k = C.k, R = C.R;
    const int shift = G * k;
    const int cmax = (1 << (cv.geom[inst].B - k)) - 1;
    const float bmul = C.band_mul, badd = C.band_add;
    const float far32 = C.far32;
    const double far64 = C.far64;
    const int32_t skip_below = max(rho_skip, C.skip);
    const unsigned long long hb = ib ? ((unsigned long long)inst << S) : 0ull;

    for_chunk_cells<G>(scode, I, p0, end, S, ib, shift, lane, [&](uint32_t first,
                                                                   unsigned long long cell) {
      uint32_t c0[G];
      unmorton<G>(cell, c0);
      Union<G> u;
      block_union<G>(c0, R, cmax, u);
      const int nr = union_runs<G>(u, hkeys, hvals, hmask, hb, n, lane, rt);
      const uint32_t T = rt.pre[nr];
      const uint32_t m = own_run_length(rt, nr, first, lane);
      for (uint32_t qbase = 0; qbase < m; qbase += 32u * kQB) {
        const uint32_t mq = min(m - qbase, 32u * kQB);
        const int L = lanes_per_query(mq);
        const int nqb = mq >= 32 ? (int)((mq + 31u) / 32u) : 1;
        const int sub = lane & (L - 1);
        uint32_t qi[kQB];
        bool has[kQB], act[kQB];
        Pt<DP> x[kQB];
        unsigned long long K[kQB];
        float s1[kQB], s2[kQB];
        uint32_t o1[kQB];
        double e1[kQB];
#pragma unroll
        for (int b = 0; b < kQB; ++b) {
          qi[b] = qbase + (uint32_t)(b * 32 + lane / L);
          has[b] = b < nqb && qi[b] < m;
          const uint32_t pq = first + (has[b] ? qi[b] : 0u);
          x[b] = load_pt<DP>(spts, pq);
          K[b] = has[b] ? skey[pq] : ~0ull;
          act[b] = has[b] && (int32_t)(K[b] >> 32) >= skip_below;
          s1[b] = s2[b] = INFINITY;
          o1[b] = 0xffffffffu;
          e1[b] = INFINITY;
        }
        // a skipped query keeps K = ~0: no candidate is above it
#pragma unroll
        for (int b = 0; b < kQB; ++b)
          if (!act[b]) K[b] = ~0ull;
        for (uint32_t w0 = 0; w0 < T; w0 += CAP) {
          const uint32_t w1 = min(T, w0 + (uint32_t)CAP);
          const int nw = (int)(w1 - w0);
          __syncwarp();
          stage_runs<DP, true>(rt, nr, w0, w1, spts, skey, wpts, wkey, lane);
          __syncwarp();
#pragma unroll 2
          for (int c = sub; c < nw; c += L) {
            const Pt<DP> y = window_pt<DP>(wpts, (uint32_t)c);
            const unsigned long long kc = wkey[c];
            const uint32_t id = key_id(kc);
#pragma unroll
            for (int b = 0; b < kQB; ++b) {
              if (b < nqb) {
                if constexpr (F64) {
                  if (kc > K[b]) {
                    const double v = dist64<DP, ND>(x[b], y);
                    if (v < e1[b] || (v == e1[b] && id < o1[b])) {
                      e1[b] = v;
                      o1[b] = id;
                    }
                  }
                } else {
                  const float v = kc > K[b] ? dist32<DP, ND>(x[b], y) : INFINITY;
                  s2[b] = fminf(s2[b], fmaxf(s1[b], v));
                  o1[b] = v < s1[b] ? id : o1[b];
                  s1[b] = fminf(s1[b], v);
                }
              }
            }
          }
        }
        // combine the L lanes of each query, then settle or queue it
#pragma unroll
        for (int b = 0; b < kQB; ++b) {
          if (b >= nqb) break;  // warp-uniform
          for (int o = L >> 1; o > 0; o >>= 1) {
            if constexpr (F64) {
              const double v = __shfl_xor_sync(kFull, e1[b], o);
              const uint32_t vo = __shfl_xor_sync(kFull, o1[b], o);
              if (v < e1[b] || (v == e1[b] && vo < o1[b])) {
                e1[b] = v;
                o1[b] = vo;
              }
            } else {
              const float b1 = __shfl_xor_sync(kFull, s1[b], o);
              const float b2 = __shfl_xor_sync(kFull, s2[b], o);
              const uint32_t bo = __shfl_xor_sync(kFull, o1[b], o);
              s2[b] = fminf(fminf(s2[b], b2), fmaxf(s1[b], b1));
              o1[b] = b1 < s1[b] ? bo : o1[b];
              s1[b] = fminf(s1[b], b1);
            }
          }
          const bool mine = has[b] && sub == 0;
          const uint32_t pq = first + qi[b];
          bool settled = false;
          if (mine && act[b]) {
            const uint32_t id = key_id(K[b]);
            if constexpr (F64) {
              settled = o1[b] != 0xffffffffu && e1[b] < far64;
              if (settled) {
                lambda[id] = (int32_t)(o1[b] - (uint32_t)I.out);
                delta[id] = sqrt(e1[b]);
              }
            } else if (o1[b] != 0xffffffffu) {
              const float bnd = band_of_cell(s1[b], bmul, badd);
              settled = bnd < far32 && s2[b] > bnd;
              if (settled) {
                const uint32_t o = o1[b] - (uint32_t)I.out;
                lambda[id] = (int32_t)o;
                delta[id] = sqrt(dist64<DP>(x[b], caller_pt<DP>(pts, dtype, I.coord, I.d, o)));
              }
            }
          } else if (mine) {
            const uint32_t id = key_id(skey[pq]);
            lambda[id] = -1;
            delta[id] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: skipped
          }
          const bool push = mine && act[b] && !settled;
          const unsigned pm = __ballot_sync(kFull, push);
          uint32_t base = 0;
          if (lane == 0 && pm) base = atomicAdd(&ctr->queue_n, (unsigned)__popc(pm));
          base = __shfl_sync(kFull, base, 0);
          if (push) {
            const uint32_t slot = base + __popc(pm & lanemask_lt);
            q.pos[slot] = pq;
            if constexpr (F64) q.s1d[slot] = e1[b];
            else q.s1[slot] = s1[b];
          }
        }
      }
    });
  }
}

inline unsigned cell_grid(uint32_t nchunk) {
  uint64_t b = ((uint64_t)nchunk + kCellWarps - 1) / kCellWarps;
  const uint64_t cap = (uint64_t)sm_count() * 64u;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <int DP, int G>
void density_cell_dg(bool fp64, const float* spts, const unsigned long long* scode,
                     const uint32_t* sid, const ClassView& cv, const CutGeom* cuts,
                     const HashInfo* hi, const unsigned long long* hkeys, const uint2* hvals,
                     int32_t* rho_out, unsigned long long* skey, Counters* ctr, cudaStream_t st) {
  const unsigned grid = cell_grid(cv.nchunk);
  if (fp64)
    k_density_cell<DP, G, true><<<grid, kCellThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys,
                                                              hvals, rho_out, skey, ctr);
  else
    k_density_cell<DP, G, false><<<grid, kCellThreads, 0, st>>>(spts, scode, sid, cv, cuts, hi, hkeys,
                                                               hvals, rho_out, skey, ctr);
}

template <int DP, int G>
void near_cell_dg(bool fp64, const float* spts, const unsigned long long* scode,
                  const unsigned long long* skey, const ClassView& cv, int32_t rho_skip,
                  const void* pts, int dtype, const CutGeom* cuts, const HashInfo* hi,
                  const unsigned long long* hkeys, const uint2* hvals, int32_t* lambda,
                  double* delta, FarQueue q, Counters* ctr, cudaStream_t st) {
  const unsigned grid = cell_grid(cv.nchunk);
  if (fp64)
    k_dep_near_cell<DP, G, true><<<grid, kCellThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                               dtype, cuts, hi, hkeys, hvals, lambda,
                                                               delta, q, ctr);
  else
    k_dep_near_cell<DP, G, false><<<grid, kCellThreads, 0, st>>>(spts, scode, skey, cv, rho_skip, pts,
                                                                dtype, cuts, hi, hkeys, hvals, lambda,
                                                                delta, q, ctr);
}

}  // namespace

void launch_density_cell(int dp, int g, bool fp64, const float* spts,
                         const unsigned long long* scode, const uint32_t* sid, const ClassView& cv,
                         const CutGeom* cuts, const HashInfo* hi, const unsigned long long* hkeys,
                         const uint2* hvals, int32_t* rho_out, unsigned long long* skey,
                         Counters* ctr, cudaStream_t st) {
  if (cv.N == 0) return;
  if (g == 1) density_cell_dg<2, 1>(fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, st);
  else if (g == 2) density_cell_dg<2, 2>(fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, st);
  else if (g == 3) density_cell_dg<4, 3>(fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, st);
  else if (dp == 4) density_cell_dg<4, 4>(fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, st);
  else density_cell_dg<8, 4>(fp64, spts, scode, sid, cv, cuts, hi, hkeys, hvals, rho_out, skey, ctr, st);
  count_launches(1);
}

void launch_dep_near_cell(int dp, int g, bool fp64, const float* spts,
                          const unsigned long long* scode, const unsigned long long* skey,
                          const ClassView& cv, int32_t rho_skip, const void* pts, int dtype,
                          const CutGeom* cuts, const HashInfo* hi,
                          const unsigned long long* hkeys, const uint2* hvals, int32_t* lambda,
                          double* delta, FarQueue q, Counters* ctr, cudaStream_t st) {
  if (cv.N == 0) return;
  if (g == 1) near_cell_dg<2, 1>(fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (g == 2) near_cell_dg<2, 2>(fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (g == 3) near_cell_dg<4, 3>(fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, st);
  else if (dp == 4) near_cell_dg<4, 4>(fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, st);
  else near_cell_dg<8, 4>(fp64, spts, scode, skey, cv, rho_skip, pts, dtype, cuts, hi, hkeys, hvals, lambda, delta, q, ctr, st);
  count_launches(1);
}

}  // namespace dpc
