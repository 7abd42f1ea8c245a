// tree.cu -- binary radix tree over the Morton-sorted points, with the
// largest order key of every subtree.
//
// This is the GPU form of the paper's priority search kd-tree (Section 4.1):
// every node knows the highest-priority key below it, so a query for the
// nearest point of higher priority skips any subtree whose maximum key is not
// above its own (the pruning of Section 4.1.2).  The tree itself is built in
// parallel from the sorted codes, one internal node per thread (Karras, HPG
// 2012); equal codes are split by their sorted position.  Its shape depends only
// on the points, so it is built once per binning; the keys are recomputed for
// every cutoff by one bottom-up pass.  One tree covers a whole class: the
// instance field heads the sort key, so each instance's points are exactly
// the leaves of one internal node (its root).
#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 256;

// Length of the common prefix of the (code, position) strings of sorted
// points i and j; -1 when j is out of range.
__device__ __forceinline__ int prefix_len(const unsigned long long* __restrict__ code, uint32_t n,
                                          int i, int j) {
  if (j < 0 || j >= (int)n) return -1;
  unsigned long long a = code[i], b = code[j];
  if (a != b) return __clzll((long long)(a ^ b));
  return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_tree_build(const unsigned long long* __restrict__ code, ClassView cv,
                             Node* __restrict__ nodes, uint32_t* __restrict__ leaf_parent,
                             uint32_t* __restrict__ root) {
  const uint32_t n = cv.N;
  const int S = cv.cls->S, ib = cv.cls->ib;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t + 1 < n; t += gridDim.x * blockDim.x) {
    const int i = (int)t;
    const int dir = (prefix_len(code, n, i, i + 1) - prefix_len(code, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = prefix_len(code, n, i, i - dir);
    int lmax = 2;
    while (prefix_len(code, n, i, i + lmax * dir) > dmin) lmax <<= 1;
    int l = 0;
    for (int s = lmax >> 1; s >= 1; s >>= 1)
      if (prefix_len(code, n, i, i + (l + s) * dir) > dmin) l += s;
    const int j = i + l * dir;
    const int dnode = prefix_len(code, n, i, j);
    int split = 0;
    int step = l;
    do {
      step = (step + 1) >> 1;
      const int ns = split + step;
      if (ns < l && prefix_len(code, n, i, i + ns * dir) > dnode) split = ns;
    } while (step > 1);
    const int gamma = i + split * dir + (dir < 0 ? -1 : 0);
    const int lo = i < j ? i : j;
    const int hi = i < j ? j : i;
    const uint32_t left = (lo == gamma) ? ((uint32_t)gamma | kLeafBit) : (uint32_t)gamma;
    const uint32_t right = (hi == gamma + 1) ? ((uint32_t)(gamma + 1) | kLeafBit) : (uint32_t)(gamma + 1);
    nodes[i].left = left;
    nodes[i].right = right;
    if (left & kLeafBit) {
      leaf_parent[left & ~kLeafBit] = (uint32_t)i;
    } else {
      nodes[left].parent = (uint32_t)i;
      nodes[left].pend = (uint32_t)j;
      nodes[left].sib = right;
      nodes[left].side = 0u;
    }
    if (right & kLeafBit) {
      leaf_parent[right & ~kLeafBit] = (uint32_t)i;
    } else {
      nodes[right].parent = (uint32_t)i;
      nodes[right].pend = (uint32_t)j;
      nodes[right].sib = left;
      nodes[right].side = 1u;
    }
    // the node whose leaves are exactly one instance is that instance's root
    const uint32_t inst = key_inst(code[lo], S, ib);
    if (inst < cv.ninst) {
      const InstDev I = cv.instance(inst);
      if ((uint32_t)lo == I.start && (uint32_t)hi + 1 == I.start + I.n) root[inst] = (uint32_t)i;
    }
  }
}

__global__ void k_root_parent(Node* nodes) { nodes[0].parent = 0u; }

// Bottom-up pass: the second child to arrive at a node computes its largest
// key and, on the first pass after a binning, its bounding box over all DP
// coordinates, and writes both into its parent's child record (dpc_device.cuh;
// a leaf's key is its point's and its box the point itself).

// Writes the summary of child `side` of node `node` into its record.
template <int DP, bool BOX>
__device__ __forceinline__ void put_child(float* nrec, uint32_t node, int side, unsigned long long key,
                                          const float* lo, const float* hi) {
  constexpr int W = rec_words<DP>();
  float* r = nrec + (size_t)node * W;
  __stcg(reinterpret_cast<unsigned long long*>(r + 4 + 2 * side), key);
  if constexpr (BOX) {
    float4* b = reinterpret_cast<float4*>(r + 8 + 2 * DP * side);
#pragma unroll
    for (int k = 0; k < DP / 2; ++k) {
      const float v0 = (4 * k < DP) ? lo[4 * k] : hi[4 * k - DP];
      const float v1 = (4 * k + 1 < DP) ? lo[4 * k + 1] : hi[4 * k + 1 - DP];
      const float v2 = (4 * k + 2 < DP) ? lo[4 * k + 2] : hi[4 * k + 2 - DP];
      const float v3 = (4 * k + 3 < DP) ? lo[4 * k + 3] : hi[4 * k + 3 - DP];
      __stcg(b + k, make_float4(v0, v1, v2, v3));
    }
  }
}

// Reads the summary of child `side` of node `node` back from its record
// (written by another thread's walk before its release).
template <int DP, bool BOX>
__device__ __forceinline__ void get_child(const float* nrec, uint32_t node, int side,
                                          unsigned long long& key, float* lo, float* hi) {
  constexpr int W = rec_words<DP>();
  const float* r = nrec + (size_t)node * W;
  key = __ldcg(reinterpret_cast<const unsigned long long*>(r + 4 + 2 * side));
  if constexpr (BOX) {
    const float4* b = reinterpret_cast<const float4*>(r + 8 + 2 * DP * side);
    float v[2 * DP];
#pragma unroll
    for (int k = 0; k < DP / 2; ++k) {
      const float4 q = __ldcg(b + k);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
#pragma unroll
    for (int a = 0; a < DP; ++a) {
      lo[a] = v[a];
      hi[a] = v[DP + a];
    }
  }
}

// A leaf's summary: its point's key, and (BOX) the point as its box.
template <int DP, bool BOX>
__device__ __forceinline__ void leaf_summary(uint32_t c, const unsigned long long* __restrict__ skey,
                                             const float* __restrict__ spts, unsigned long long& key,
                                             float* lo, float* hi) {
  const uint32_t t = c & ~kLeafBit;
  key = skey[t];
  if constexpr (BOX) {
    const Pt<DP> p = load_pt<DP>(spts, t);
#pragma unroll
    for (int a = 0; a < DP; ++a) lo[a] = hi[a] = p.x[a];
  }
}

// Arrival counter with acquire-release semantics at GPU scope: the first
// child to arrive publishes its subtree's results (release), the second reads
// them after its own increment (acquire), without full fences.
__device__ __forceinline__ uint32_t arrive(uint32_t* counter) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(counter) : "memory");
  return old;
}

// One thread per node for the bottom-up walks: a thread that strode over
// several nodes would run their walks one after another, each a chain of
// dependent loads; with one node per thread every walk starts at once and
// the blocks are scheduled as earlier ones retire.
// (blocks of 128: a block holds its slot until its longest walk ends, so
// smaller blocks free slots sooner, larger ones keep more meetings local; on
// c3 0.84 ms against 0.85 with 64, 0.89 with 256 and 0.93 with 512)
constexpr int kUpThreads = 128;

// Arrival counter in shared memory, acquire-release at block scope.
__device__ __forceinline__ uint32_t arrive_cta(uint32_t* counter) {
  uint32_t old;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(counter);
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(a) : "memory");
  return old;
}

// One thread per internal node whose two children are both leaves (the
// bottom of the tree: about a third of the nodes).  It computes that node and
// walks up, carrying the node's results in registers.  A parent whose other
// child is a leaf is computed at once; only at a parent with two internal
// children do the two walks meet, and the second to arrive continues with
// the first's results.  The internal nodes below a node with leaf range
// [lo, hi] are numbered within [lo, hi], so when that range lies inside the
// block's own 128 node numbers both walks run in this block: they meet
// through a shared-memory counter and summary slots (block-scope ordering),
// and only nodes whose range crosses a block boundary (a few percent) take
// the global acq_rel counter.  Every node's record gets its children's
// indices, keys and (BOX) boxes on the way.
template <int DP, bool BOX>
__global__ void __launch_bounds__(kUpThreads) k_tree_up(const unsigned long long* __restrict__ skey,
                                                        const float* __restrict__ spts, uint32_t n,
                                                        const Node* __restrict__ nodes,
                                                        uint32_t* visit, float* nrec) {
  constexpr int W = rec_words<DP>();
  constexpr int SB = BOX ? 2 * DP : 1;
  __shared__ uint32_t s_cnt[kUpThreads];
  __shared__ unsigned long long s_key[2 * kUpThreads];  // [node - base][side]
  __shared__ float s_box[2 * kUpThreads * SB];          // [node - base][side][lo | hi]
  const uint32_t base = blockIdx.x * kUpThreads;
  s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  // the launch has one thread per internal node (grid_all)
  const uint32_t t = base + threadIdx.x;
  if (t + 1 >= n) return;
  uint32_t node = t;
  const uint32_t l0 = nodes[node].left, r0 = nodes[node].right;
  if (!((l0 & kLeafBit) && (r0 & kLeafBit))) return;
  // this node from its two leaves
  unsigned long long key;
  float lo[DP], hi[DP];
  {
    unsigned long long kr;
    float lo2[DP], hi2[DP];
    leaf_summary<DP, BOX>(l0, skey, spts, key, lo, hi);
    leaf_summary<DP, BOX>(r0, skey, spts, kr, lo2, hi2);
    __stcg(reinterpret_cast<uint2*>(nrec + (size_t)node * W), make_uint2(l0, r0));
    put_child<DP, BOX>(nrec, node, 0, key, lo, hi);
    put_child<DP, BOX>(nrec, node, 1, kr, lo2, hi2);
    key = key > kr ? key : kr;
    if constexpr (BOX) {
#pragma unroll
      for (int a = 0; a < DP; ++a) {
        lo[a] = fminf(lo[a], lo2[a]);
        hi[a] = fmaxf(hi[a], hi2[a]);
      }
    }
  }
  for (uint32_t depth = 0; depth < 2u * n + 64u; ++depth) {
    if (node == 0u) break;
    // sibling, side, parent and the far end of the parent's leaf range
    // (k_tree_build)
    const uint2 ps = *reinterpret_cast<const uint2*>(&nodes[node].sib);
    const uint2 pp = *reinterpret_cast<const uint2*>(&nodes[node].parent);
    const uint32_t par = pp.x;
    const int side = (int)(ps.y & 1u);
    const uint32_t sib = ps.x;
    const uint32_t pl = side == 0 ? node : sib, pr = side == 0 ? sib : node;
    unsigned long long ks;
    float lo2[DP], hi2[DP];
    if (sib & kLeafBit) {
      put_child<DP, BOX>(nrec, par, side, key, lo, hi);
      leaf_summary<DP, BOX>(sib, skey, spts, ks, lo2, hi2);
      put_child<DP, BOX>(nrec, par, 1 - side, ks, lo2, hi2);
    } else {
      const uint32_t plo = par < pp.y ? par : pp.y, phi = par < pp.y ? pp.y : par;
      if (plo >= base && phi < base + kUpThreads) {
        // both walks in this block: the summary into this side's slot, then
        // the block-scope arrival; the record in global memory is written
        // after it (read only by later launches)
        const uint32_t k = par - base;
        s_key[2 * k + side] = key;
        if constexpr (BOX) {
#pragma unroll
          for (int a = 0; a < DP; ++a) {
            s_box[(2 * k + side) * SB + a] = lo[a];
            s_box[(2 * k + side) * SB + DP + a] = hi[a];
          }
        }
        const uint32_t old = arrive_cta(&s_cnt[k]);
        put_child<DP, BOX>(nrec, par, side, key, lo, hi);
        if (old == 0u) break;  // the sibling's walk continues
        ks = s_key[2 * k + 1 - side];
        if constexpr (BOX) {
#pragma unroll
          for (int a = 0; a < DP; ++a) {
            lo2[a] = s_box[(2 * k + 1 - side) * SB + a];
            hi2[a] = s_box[(2 * k + 1 - side) * SB + DP + a];
          }
        }
      } else {
        // this node's summary into the parent's record, before the release
        put_child<DP, BOX>(nrec, par, side, key, lo, hi);
        if (arrive(&visit[par]) == 0u) break;  // the sibling's walk continues
        get_child<DP, BOX>(nrec, par, 1 - side, ks, lo2, hi2);
      }
    }
    // the parent from this node (registers) and its sibling
    __stcg(reinterpret_cast<uint2*>(nrec + (size_t)par * W), make_uint2(pl, pr));
    key = key > ks ? key : ks;
    if constexpr (BOX) {
#pragma unroll
      for (int a = 0; a < DP; ++a) {
        lo[a] = fminf(lo[a], lo2[a]);
        hi[a] = fmaxf(hi[a], hi2[a]);
      }
    }
    node = par;
  }
}

inline unsigned grid_for(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > sm_count() * 16u) b = sm_count() * 16u;
  return (unsigned)b;
}

inline unsigned grid_all(uint64_t n) {
  uint64_t b = (n + kUpThreads - 1) / kUpThreads;
  if (b < 1) b = 1;
  if (b > 0x7fffffffull) b = 0x7fffffffull;
  return (unsigned)b;
}

}  // namespace

void launch_tree_build(const unsigned long long* scode, const ClassView& cv, Node* nodes,
                       uint32_t* leaf_parent, uint32_t* root, cudaStream_t st) {
  cudaMemsetAsync(root, 0xff, sizeof(uint32_t) * cv.ninst, st);
  if (cv.N < 2) return;
  k_tree_build<<<grid_for(cv.N - 1), kThreads, 0, st>>>(scode, cv, nodes, leaf_parent, root);
  k_root_parent<<<1, 1, 0, st>>>(nodes);
  count_launches(2);
}

template <int DP>
void tree_up_dp(const unsigned long long* skey, const float* spts, uint32_t n, Node* nodes,
                const uint32_t* leaf_parent, uint32_t* visit, float* nbox, bool boxes,
                cudaStream_t st) {
  (void)leaf_parent;
  if (boxes)
    k_tree_up<DP, true><<<grid_all(n - 1), kUpThreads, 0, st>>>(skey, spts, n, nodes, visit, nbox);
  else
    k_tree_up<DP, false><<<grid_all(n - 1), kUpThreads, 0, st>>>(skey, spts, n, nodes, visit, nbox);
}

void launch_tree_maxkey(const unsigned long long* skey, const float* spts, int dp, uint32_t n,
                        Node* nodes, const uint32_t* leaf_parent, uint32_t* visit, float* nrec,
                        bool boxes, cudaStream_t st) {
  if (n < 2) return;
  cudaMemsetAsync(visit, 0, sizeof(uint32_t) * (n - 1), st);
  if (dp == 2) tree_up_dp<2>(skey, spts, n, nodes, leaf_parent, visit, nrec, boxes, st);
  else if (dp == 4) tree_up_dp<4>(skey, spts, n, nodes, leaf_parent, visit, nrec, boxes, st);
  else tree_up_dp<8>(skey, spts, n, nodes, leaf_parent, visit, nrec, boxes, st);
  count_launches(1);
}

}  // namespace dpc
