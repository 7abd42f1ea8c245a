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
// every cutoff by one bottom-up pass.
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

__global__ void k_tree_build(const unsigned long long* __restrict__ code, uint32_t n,
                             const GridGeom* __restrict__ geom, Node* __restrict__ nodes,
                             uint32_t* __restrict__ leaf_parent) {
  const int nbits = geom->nbits;
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
    Node nd;
    nd.left = (lo == gamma) ? ((uint32_t)gamma | kLeafBit) : (uint32_t)gamma;
    nd.right = (hi == gamma + 1) ? ((uint32_t)(gamma + 1) | kLeafBit) : (uint32_t)(gamma + 1);
    nd.maxkey = 0ull;
    nd.code = code[lo];
    // prefix inside the nbits-bit code (the top 64 - nbits bits are always 0)
    int pl = dnode - (64 - nbits);
    nd.plen = (uint32_t)(pl < 0 ? 0 : (pl > nbits ? nbits : pl));
    nd.parent = (uint32_t)i;  // root keeps itself; children overwrite below
    nodes[i].left = nd.left;
    nodes[i].right = nd.right;
    nodes[i].maxkey = nd.maxkey;
    nodes[i].code = nd.code;
    nodes[i].plen = nd.plen;
    if (nd.left & kLeafBit) leaf_parent[nd.left & ~kLeafBit] = (uint32_t)i;
    else nodes[nd.left].parent = (uint32_t)i;
    if (nd.right & kLeafBit) leaf_parent[nd.right & ~kLeafBit] = (uint32_t)i;
    else nodes[nd.right].parent = (uint32_t)i;
  }
}

__global__ void k_root_parent(Node* nodes) { nodes[0].parent = 0u; }

// Bottom-up maximum key: the second child to arrive at a node computes it.
__global__ void k_tree_maxkey(const unsigned long long* __restrict__ skey, uint32_t n,
                              Node* nodes, const uint32_t* __restrict__ leaf_parent,
                              uint32_t* visit) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    uint32_t node = leaf_parent[t];
    for (uint32_t depth = 0; depth < 2u * n + 64u; ++depth) {
      __threadfence();
      if (atomicAdd(&visit[node], 1u) == 0u) break;  // first arrival: the sibling continues
      __threadfence();
      const uint32_t l = nodes[node].left, r = nodes[node].right;
      const unsigned long long kl =
          (l & kLeafBit) ? skey[l & ~kLeafBit] : __ldcg(&nodes[l].maxkey);
      const unsigned long long kr =
          (r & kLeafBit) ? skey[r & ~kLeafBit] : __ldcg(&nodes[r].maxkey);
      __stcg(&nodes[node].maxkey, kl > kr ? kl : kr);
      if (node == 0u) break;
      node = nodes[node].parent;
    }
  }
}

inline unsigned grid_for(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152u * 16u) b = 152u * 16u;
  return (unsigned)b;
}

}  // namespace

void launch_tree_build(const unsigned long long* scode, uint32_t n, const GridGeom* geom,
                       Node* nodes, uint32_t* leaf_parent, cudaStream_t st) {
  if (n < 2) return;
  k_tree_build<<<grid_for(n - 1), kThreads, 0, st>>>(scode, n, geom, nodes, leaf_parent);
  k_root_parent<<<1, 1, 0, st>>>(nodes);
  count_launches(2);
}

void launch_tree_maxkey(const unsigned long long* skey, uint32_t n, Node* nodes,
                        const uint32_t* leaf_parent, uint32_t* visit, cudaStream_t st) {
  if (n < 2) return;
  cudaMemsetAsync(visit, 0, sizeof(uint32_t) * (n - 1), st);
  k_tree_maxkey<<<grid_for(n), kThreads, 0, st>>>(skey, n, nodes, leaf_parent, visit);
  count_launches(1);
}

}  // namespace dpc
