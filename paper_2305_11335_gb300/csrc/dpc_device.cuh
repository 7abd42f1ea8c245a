// dpc_device.cuh -- device-side data structures and helpers shared by the
// kernels of the exact DPC library (sm_103a).
//
// Work is organised in classes: the instances of a batch that share the
// padded dimension DP and the gridded dimension g are processed together, one
// launch per kernel for the whole class.  Their points are concatenated
// (instance i owns positions [start_i, start_i + n_i)) and sorted by the key
// (i << S) | Morton code, so every instance stays a contiguous range of the
// sorted order and each of its grid cells a contiguous run inside it.
//
// Layout in HBM for one class of N points (see the kernels for who writes
// what):
//   codes      u64[N]   sort key of each point, (instance << S) | Morton code
//   spts       float[N][DP] points in key order, zero padded to DP = 2/4/8
//   sid        u32[N]   output index of each sorted point (the instance's
//                       offset in the caller's arrays + its id there)
//   skey       u64[N]   order key of each sorted point, (rho << 32) | ~sid
//   hash       u64[T] keys + uint2[T] (start, end) of each occupied cell of
//              the density grid level of every instance, open addressing
//   tree       Node[N-1] binary radix tree over the sorted keys; instance i
//              is the subtree below root[i]
//
// The grid of an instance: a fine uniform grid of 2^B cells per gridded axis
// (the first g = min(d, 4) coordinates) covers its bounding box; a point's
// fine index is floor((x - org) / f).  Level k of the grid merges 2^k fine
// cells per axis; since the Morton code interleaves the axes, every level-k
// cell is the contiguous run of sorted points sharing key >> (g*k) (the
// instance field sits above every code bit).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpc {

constexpr int kMaxDim = 8;
constexpr int kMaxBits = 21;              // fine-grid bits per axis (k_setup_geom)
constexpr int kMaxGrid = 4;               // gridded coordinates

// Gridded coordinates of a d-dimensional instance.
__host__ __device__ __forceinline__ int grid_dims(int d) { return d < kMaxGrid ? d : kMaxGrid; }
constexpr uint64_t kEmpty = ~0ull;        // empty hash slot (codes are < 2^63)
constexpr uint32_t kLeafBit = 0x80000000u;

// status bits recorded on the device
enum : int {
  kStatusBadCoord = 1,   // NaN/Inf or out-of-range coordinate
  kStatusHashFull = 2,   // hash probe limit reached (cannot happen at load <= 1/2)
  kStatusStack = 4,      // tree traversal stack overflow
  kStatusCycle = 8,      // dependent pointers did not converge to roots
  kStatusIndex = 16,     // an internal index failed its bounds check (a bug)
  kStatusTimeout = 32,   // a bounded wait for the tensor core gave up
  kStatusQuery = 64      // a query names an instance outside the batch
};

// Per-instance grid geometry, written by the setup kernel from the bounding box.
struct GridGeom {
  double org[kMaxGrid];  // bounding-box minimum of the gridded axes
  double f;          // fine cell side
  double inv_f;      // 1 / f
  float f2;          // f*f rounded down (for lower bounds)
  int g;             // gridded axes
  int B;             // fine-grid bits per axis
  int nbits;         // g * B
  int* status;       // the workspace's device status word (kStatus* bits)
  uint32_t bbox_ord[2 * kMaxGrid];  // ordered-uint min (0..3) and max (4..7) accumulators
};

// Per-class sort-key layout and status.
struct ClassGeom {
  int S;         // bit position of the instance field: max over instances of g*B
  int ib;        // bits of the instance field (0 for a single instance)
  int bcap;      // largest B allowed, so that the key stays below 2^63
  int pad;
  int* status;   // the workspace's device status word
};

// One instance of a class (device copy of the host's description).
struct InstDev {
  uint32_t start;      // first position of the instance in the class's arrays
  uint32_t n;          // points
  uint64_t out;        // offset of the instance in the caller's result arrays
  uint64_t coord;      // element offset of its coordinates in the caller's pts
  int32_t d;           // dimension
  uint32_t chunk0;     // first 32-point chunk of the instance
  uint32_t row;        // the instance's index in the caller's batch
  uint32_t pad;
};

// Labelling thresholds of one (instance, cutoff) (same layout as dpc_params).
struct LabelParams {
  int32_t rho_noise;
  int32_t rho_min;
  double delta_min;
};

constexpr uint32_t kNoNode = 0xffffffffu;  // no internal node (instance of one point)

// Hash-table size of one class and cutoff.
struct HashInfo {
  uint32_t m;          // occupied cells (all instances)
  uint32_t hmask;      // table size - 1
  uint32_t work;       // work counter of kernels that take items one by one
  uint32_t npieces;    // entries of the piece list (tensor-core density)
};

// What a kernel needs to know about the class it works on.  A chunk is up to
// 32 consecutive positions of one instance; chunk c of a single-instance
// class holds positions 32c .. 32c+31, so it needs no tables.
struct ClassView {
  uint32_t N;                     // points of the class
  uint32_t ninst;                 // instances
  uint32_t nchunk;                // chunks
  const InstDev* inst;            // [ninst], or null for a single instance (`one`)
  const uint32_t* chunk_inst;     // [nchunk] instance of each chunk (null: single)
  const uint32_t* chunk_pos;      // [nchunk] first position of each chunk
  InstDev one;                    // the single instance when inst is null
  GridGeom* geom;                 // [ninst]
  ClassGeom* cls;

  __device__ __forceinline__ InstDev instance(uint32_t i) const { return inst ? inst[i] : one; }
  // instance, first position and end of the instance's range for chunk c
  __device__ __forceinline__ void chunk(uint32_t c, uint32_t& i, uint32_t& p0, uint32_t& end) const {
    if (chunk_inst) {
      i = chunk_inst[c];
      p0 = chunk_pos[c];
      const InstDev I = inst[i];
      end = I.start + I.n;
    } else {
      i = 0;
      p0 = c * 32u;
      end = N;
    }
  }
};

// Instance field and Morton code of a sort key.
__device__ __forceinline__ uint32_t key_inst(unsigned long long key, int S, int ib) {
  return ib ? (uint32_t)(key >> S) : 0u;
}
__device__ __forceinline__ unsigned long long key_code(unsigned long long key, int S, int ib) {
  return ib ? (key & ((1ull << S) - 1ull)) : key;
}
// 8-bit radix passes that sort keys of S + ib bits.
__host__ __device__ __forceinline__ int sort_passes(int S, int ib) { return (S + ib + 7) / 8; }

// Per (instance, cutoff) parameters.  Fields marked [host] are filled before
// the launch; the others by the setup kernels.
struct CutGeom {
  double dc;          // d_cut                                           [host]
  double dc2;         // fl64(d_cut * d_cut): the density predicate      [host]
  float t_in;         // float32 filter: s32 <= t_in  => s64 <= dc2      [host]
  float t_out;        // float32 filter: s32 >  t_out => s64 >  dc2      [host]
  float band_mul;     // float32 ambiguity band: s_b > s_a*band_mul+band_add
  float band_add;     //   => s64_b > s64_a                              [host]
  int k;              // grid level of the density / near-dependent search
  int R;              // neighbourhood radius in level-k cells
  float prune_fine;   // density: a cell whose squared lower bound, in fine
                      //   units, exceeds this holds no point within d_cut
  float far32;        // dependent: a float32 winner band below this is
  double far64;       //   settled by the (2R+1)^g block (float / double forms)
  uint32_t m;         // occupied level-k cells
  uint32_t hmask;     // hash table size - 1
  int32_t skip;       // dependent: points with rho < skip are skipped   [host]
  int32_t pad;
};

// Counters for dpc_get_stats.
struct Counters {
  unsigned long long band_pairs;
  unsigned long long far_queries;
  unsigned long long exact_rescans;
  unsigned long long far_nodes;   // tree nodes expanded by far queries
  unsigned long long far_wide_queries;  // far queries that needed the second round
  unsigned long long pairs;       // density: (query, candidate) pairs evaluated
  unsigned int far_nodes_max;     // most tree nodes expanded by one far query
  unsigned int queue_n;           // dependent far-query queue length
  unsigned int queue2_n;          // far queries passed to the second round
  unsigned int pad;
};

// One internal node of the binary radix tree over the sorted keys.
struct __align__(8) Node {
  uint32_t left, right;   // child index; kLeafBit marks a leaf (sorted point)
  uint32_t sib;           // the parent's other child (kLeafBit: a sorted point)
  uint32_t side;          // 0: this node is its parent's left child, 1: right
  uint32_t parent;        // parent internal node (root: itself)
  uint32_t pend;          // the parent's number is one end of its leaf range; this is the other
};

// Child records of the radix tree (tree.cu): internal node i keeps in one
// 16-byte-aligned record of rec_words<DP>() words what a search needs about
// both its children -- their indices, their largest order keys and their
// bounding boxes (a leaf's box is its point) -- so that expanding a node is
// one load instead of a chain of dependent ones.
//   words 0, 1                 left, right child (kLeafBit: a sorted point)
//   words 4..5, 6..7           largest order key below the left, right child
//   words 8 .. 8+2DP           box of the left child [lo(DP) | hi(DP)]
//   words 8+2DP .. 8+4DP       box of the right child
template <int DP>
constexpr int rec_words() { return 8 + 4 * DP; }
constexpr int kRecWordsMax = 8 + 4 * 8;

template <int DP>
struct ChildRec {
  uint32_t child[2];
  unsigned long long key[2];
  float lo[2][DP], hi[2][DP];
};

template <int DP>
__device__ __forceinline__ ChildRec<DP> load_rec(const float* __restrict__ nrec, uint32_t node) {
  constexpr int W = rec_words<DP>();
  const float4* r = reinterpret_cast<const float4*>(nrec) + (size_t)node * (W / 4);
  float v[W];
#pragma unroll
  for (int k = 0; k < W / 4; ++k) {
    const float4 q = __ldg(r + k);
    v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
  }
  ChildRec<DP> c;
  c.child[0] = __float_as_uint(v[0]);
  c.child[1] = __float_as_uint(v[1]);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    c.key[s] = ((unsigned long long)__float_as_uint(v[5 + 2 * s]) << 32) | __float_as_uint(v[4 + 2 * s]);
#pragma unroll
    for (int a = 0; a < DP; ++a) {
      c.lo[s][a] = v[8 + 2 * DP * s + a];
      c.hi[s][a] = v[8 + 2 * DP * s + DP + a];
    }
  }
  return c;
}

// ---------------------------------------------------------------------------
// Morton codes: axis a's bit b sits at position g*b + a.

__host__ __device__ __forceinline__ uint64_t spread2(uint64_t x) {  // 32 -> 64 bits
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact2(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x | (x >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t x) {  // 21 -> 63 bits
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x001f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x001f00000000ffffull;
  x = (x | (x >> 32)) & 0x00000000001fffffull;
  return (uint32_t)x;
}

__host__ __device__ __forceinline__ uint64_t spread4(uint64_t x) {  // 16 -> 64 bits
  x &= 0xffffull;
  x = (x ^ (x << 24)) & 0x000000ff000000ffull;
  x = (x ^ (x << 12)) & 0x000f000f000f000full;
  x = (x ^ (x << 6)) & 0x0303030303030303ull;
  x = (x ^ (x << 3)) & 0x1111111111111111ull;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact4(uint64_t x) {
  x &= 0x1111111111111111ull;
  x = (x ^ (x >> 3)) & 0x0303030303030303ull;
  x = (x ^ (x >> 6)) & 0x000f000f000f000full;
  x = (x ^ (x >> 12)) & 0x000000ff000000ffull;
  x = (x ^ (x >> 24)) & 0x000000000000ffffull;
  return (uint32_t)x;
}

template <int G>
__host__ __device__ __forceinline__ uint64_t morton(const uint32_t* c) {
  if constexpr (G == 1) return c[0];
  else if constexpr (G == 2) return spread2(c[0]) | (spread2(c[1]) << 1);
  else if constexpr (G == 3) return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
  else return spread4(c[0]) | (spread4(c[1]) << 1) | (spread4(c[2]) << 2) | (spread4(c[3]) << 3);
}
template <int G>
__host__ __device__ __forceinline__ void unmorton(uint64_t code, uint32_t* c) {
  if constexpr (G == 1) c[0] = (uint32_t)code;
  else if constexpr (G == 2) { c[0] = compact2(code); c[1] = compact2(code >> 1); }
  else if constexpr (G == 3) { c[0] = compact3(code); c[1] = compact3(code >> 1); c[2] = compact3(code >> 2); }
  else {
    c[0] = compact4(code); c[1] = compact4(code >> 1);
    c[2] = compact4(code >> 2); c[3] = compact4(code >> 3);
  }
}

// ---------------------------------------------------------------------------
// Open-addressing hash of occupied cells: key = level-k Morton code.

__device__ __forceinline__ uint32_t hash_slot(uint64_t key, uint32_t mask) {
  key ^= key >> 33;
  key *= 0xff51afd7ed558ccdull;
  key ^= key >> 33;
  key *= 0xc4ceb9fe1a85ec53ull;
  key ^= key >> 33;
  return (uint32_t)key & mask;
}

// Returns (start, end) of the cell's sorted-point run, or (0, 0) if empty.
__device__ __forceinline__ uint2 hash_find(const unsigned long long* __restrict__ keys,
                                           const uint2* __restrict__ vals, uint32_t mask,
                                           uint64_t key) {
  uint32_t h = hash_slot(key, mask);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    unsigned long long k = __ldg(keys + h);
    if (k == key) return __ldg(vals + h);
    if (k == kEmpty) break;
    h = (h + 1) & mask;
  }
  return make_uint2(0u, 0u);
}

// A cell run clipped to [0, n): the hash only holds runs of this instance, so
// the clip never changes a valid run; it keeps a corrupted one in bounds.
__device__ __forceinline__ uint2 clip_run(uint2 r, uint32_t n) {
  r.y = r.y < n ? r.y : n;
  r.x = r.x < r.y ? r.x : r.y;
  return r;
}

// ---------------------------------------------------------------------------
// Distances.

// Point coordinates padded to DP floats (DP = 2, 4 or 8).
template <int DP>
struct Pt {
  float x[DP];
};

template <int DP>
__device__ __forceinline__ Pt<DP> load_pt(const float* __restrict__ spts, uint32_t i) {
  Pt<DP> p;
  if constexpr (DP == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(spts) + i);
    p.x[0] = v.x; p.x[1] = v.y;
  } else if constexpr (DP == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(spts) + i);
    p.x[0] = v.x; p.x[1] = v.y; p.x[2] = v.z; p.x[3] = v.w;
  } else {
    const float4* q = reinterpret_cast<const float4*>(spts) + 2 * (size_t)i;
    float4 a = __ldg(q), b = __ldg(q + 1);
    p.x[0] = a.x; p.x[1] = a.y; p.x[2] = a.z; p.x[3] = a.w;
    p.x[4] = b.x; p.x[5] = b.y; p.x[6] = b.z; p.x[7] = b.w;
  }
  return p;
}

// float32 filter value: any evaluation order, contraction allowed; its error
// against the exact squared distance is covered by the bands in CutGeom.
// Coordinates that can be nonzero in a class of padded dimension DP with G
// gridded axes: every instance of a class with fewer than 4 gridded axes has
// d = G (the rest is zero padding); from 4 gridded axes on, up to DP.
template <int DP, int G>
constexpr int real_dims() { return G < 4 ? G : DP; }

// ND <= DP leading coordinates (the others are padding zeros that add 0).
template <int DP, int ND = DP>
__device__ __forceinline__ float dist32(const Pt<DP>& a, const Pt<DP>& b) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    float t = a.x[k] - b.x[k];
    s = fmaf(t, t, s);
  }
  return s;
}

// The canonical binary64 squared distance: t_k = x_k - y_k, s = ((t0*t0 + t1*t1) + ...)
// in increasing k, each step rounded to nearest, never contracted.  Padding
// coordinates are zero and add exactly 0.
template <int DP, int ND = DP>
__device__ __forceinline__ double dist64(const Pt<DP>& a, const Pt<DP>& b) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    double t = __dsub_rn((double)a.x[k], (double)b.x[k]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// ---------------------------------------------------------------------------
// Packed float32 pairs: add / mul / fma on the two float32 halves of a 64-bit
// register in one instruction (sm_100 and later), each half rounded to nearest
// exactly as the scalar operation, subnormals kept.  The segment kernels
// evaluate dist32 for two candidates at once with them -- the same value bit
// for bit, in half the issue slots.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo2(f32x2 v) {
  float lo;
  asm("mov.b64 {%0, _}, %1;" : "=f"(lo) : "l"(v));
  return lo;
}
__device__ __forceinline__ float hi2(f32x2 v) {
  float hi;
  asm("mov.b64 {_, %0}, %1;" : "=f"(hi) : "l"(v));
  return hi;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// dist32 of a query against two candidates at once.  q2[k] holds the query's
// coordinate k in both halves, nc[k] the two candidates' coordinate k negated:
// t = q + (-c) rounds exactly as q - c, and s = t0*t0 (= fma(t0, t0, 0)), then
// s = fma(t_k, t_k, s) in increasing k: dist32's sequence in each half.
template <int ND>
__device__ __forceinline__ f32x2 dist32x2(const f32x2* q2, const f32x2* nc) {
  f32x2 t = add2(q2[0], nc[0]);
  f32x2 s = mul2(t, t);
#pragma unroll
  for (int k = 1; k < ND; ++k) {
    t = add2(q2[k], nc[k]);
    s = fma2(t, t, s);
  }
  return s;
}

// The next float above x (finite x): s <= x  <=>  s < next_up(x) for floats.
__device__ __forceinline__ float next_up(float x) {
  const uint32_t b = __float_as_uint(x);
  if (b == 0x80000000u) return __uint_as_float(1u);  // -0: the least positive subnormal
  return __uint_as_float((b >> 31) ? b - 1u : b + 1u);
}

// Number of negative halves of a packed pair (sign bits: fl(s - t) is
// negative exactly when s < t, for s, t not NaN).
__device__ __forceinline__ uint32_t sign_count2(f32x2 u) {
  return (__float_as_uint(lo2(u)) >> 31) + (__float_as_uint(hi2(u)) >> 31);
}

// The float32 filter band t_in < s <= t_out as one unsigned test on the bit
// pattern of s >= +0 (non-negative floats order like their bit patterns):
// (bits(s) - lo) < width.  A negative (or -0) t_in takes every s from +0 on
// (a superset: the band pass rechecks each pair exactly); NaN and values above
// t_out fall outside.
struct BandBits {
  uint32_t lo, width;
};
__device__ __forceinline__ BandBits band_bits(float t_in, float t_out) {
  const uint32_t bi = __float_as_uint(t_in);
  const uint32_t lo = (bi >> 31) ? 0u : bi + 1u;
  return BandBits{lo, __float_as_uint(t_out) + 1u - lo};
}
// min over both halves of s of bits(s) - lo: below BandBits::width iff a half
// lies in the band.
__device__ __forceinline__ uint32_t band_min2(f32x2 s, uint32_t lo) {
  return min(__float_as_uint(lo2(s)) - lo, __float_as_uint(hi2(s)) - lo);
}

// Order key: larger = higher in the total order (density, then smaller id).
__device__ __forceinline__ unsigned long long order_key(int32_t rho, uint32_t id) {
  return ((unsigned long long)(uint32_t)rho << 32) | (unsigned long long)(0xffffffffu - id);
}
__device__ __forceinline__ uint32_t key_id(unsigned long long key) {
  return 0xffffffffu - (uint32_t)key;
}

// Ordered-uint encoding of floats (monotone), for atomic min/max.
__device__ __forceinline__ uint32_t float_ord(float x) {
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord_float(uint32_t u) {
  uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(v);
#else
  float f;
  __builtin_memcpy(&f, &v, 4);
  return f;
#endif
}

__device__ __forceinline__ void set_status(int* status, int bits) { atomicOr(status, bits); }

}  // namespace dpc
