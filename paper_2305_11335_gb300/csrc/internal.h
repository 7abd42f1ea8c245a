// internal.h -- host-side launchers of the library's kernels (not part of the ABI).
//
// Every launcher works on one class (dpc_device.cuh): the instances of a call
// that share the padded dimension dp and the gridded dimension g.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpc_device.cuh"

namespace dpc {

// Streaming multiprocessors of the current device (grid caps are multiples
// of it); queried once per device.
unsigned sm_count();

// Polls a bounded device-side wait makes before it gives up: `dflt`, or the
// smaller value in the environment variable DPC_TEST_WAIT_LIMIT (tests use 0
// to make every such wait give up at once and check the recovery path).
uint32_t wait_limit(uint32_t dflt);

// Largest single device allocation the library may make (the environment
// variable DPC_WORKSPACE_LIMIT_BYTES, unset = no limit).  dev_alloc fails
// without calling cudaMalloc when a request is larger.
bool dev_alloc(void** p, size_t bytes);

// Kernels enqueued by the current call (the entry points hold the library
// lock while enqueueing, so a plain counter suffices).
extern long long g_kernel_launches;
inline void count_launches(int k) { g_kernel_launches += k; }

// Host-computed constants of one cutoff (the [host] fields of CutGeom).
struct CutHost {
  double dc, dc2;
  float t_in, t_out, band_mul, band_add;
  int32_t skip;  // dependent search: points with rho < skip are skipped
  int32_t pad;
};
CutHost make_cut_host(double d_cut, int dp);

// Cutoffs passed by value (single-instance calls that have no device copy).
constexpr int kCutChunk = 16;
struct CutArgs {
  CutHost h[kCutChunk];
};

// ---- binning (binning.cu) ---------------------------------------------------
void launch_class_init(const ClassView& cv, int g, int ib, int bcap, int* status, cudaStream_t st);
// chunk tables of a multi-instance class (InstDev::chunk0 gives each instance's first chunk)
void launch_chunks(const ClassView& cv, uint32_t* chunk_inst, uint32_t* chunk_pos, cudaStream_t st);
void launch_bbox(const void* pts, int dtype, const ClassView& cv, int g, cudaStream_t st);
// per-instance grid and per (instance, cutoff) parameters; cutoffs come from
// hc_dev ([ninst][ncut], device) or, when it is null, from hc_host (ncut <= kCutChunk)
void launch_setup(const ClassView& cv, CutGeom* cuts, int ncut, const CutHost* hc_dev,
                  const CutHost* hc_host, cudaStream_t st);
// level and block radius of one cutoff (cuts: [ninst]) again: rpref = 0 the
// default rule, rpref > 0 the finest level whose block radius is <= rpref
void launch_set_radius(const ClassView& cv, CutGeom* cuts, int rpref, cudaStream_t st);
// near-dependent search `shift` grid levels finer than the density's (0: same)
void launch_near_level(const ClassView& cv, CutGeom* cuts, int shift, cudaStream_t st);
void launch_codes(const void* pts, int dtype, const ClassView& cv, int g, unsigned long long* codes,
                  uint32_t* ids, cudaStream_t st);
void launch_gather(const void* pts, int dtype, const ClassView& cv, int dp,
                   const unsigned long long* codes_a, const unsigned long long* codes_b,
                   const uint32_t* ids_a, const uint32_t* ids_b, float* spts,
                   unsigned long long* scode, uint32_t* sid, cudaStream_t st);
// occupied level-k cells of every instance for one cutoff (cuts: [ninst]) -> hash
void launch_cells(const unsigned long long* scode, const ClassView& cv, int g, const CutGeom* cuts,
                  HashInfo* hi, unsigned long long* hkeys, uint2* hvals, uint32_t hcap,
                  cudaStream_t st);

// ---- radix sort (sort.cu) ------------------------------------------------------
constexpr uint32_t kSortTile = 4096;    // items per tile of one pass
constexpr uint32_t kSortMaxPasses = 8;  // 8-bit digits of a 64-bit key
// 32-bit words of sort scratch for n items: per tile and digit a published
// 64-bit count, the digit counts and starts of every pass, a tile counter per
// pass (and slack)
constexpr size_t sort_hist_words_for(uint64_t n) {
  return (size_t)(n ? (n + kSortTile - 1) / kSortTile : 1) * 256u * 2u +
         2u * kSortMaxPasses * 256u + kSortMaxPasses + 8u;
}
size_t sort_hist_words(uint32_t n);
// one-time kernel attribute setup (called before any stream capture)
void sort_init();
// Sorts (codes_a, ids_a) by code, LSD over the device-side pass count
// sort_passes(cls->S, cls->ib); the result lands in the _a buffers if that
// count is even, else in _b.
void launch_sort(unsigned long long* codes_a, unsigned long long* codes_b, uint32_t* ids_a,
                 uint32_t* ids_b, uint32_t n, const ClassGeom* cls, uint32_t* hist,
                 cudaStream_t st);

// ---- radix tree (tree.cu) ------------------------------------------------------
// Tree over the class's sorted keys; root[i] = the internal node whose leaves
// are exactly instance i (kNoNode for an instance of one point).
void launch_tree_build(const unsigned long long* scode, const ClassView& cv, Node* nodes,
                       uint32_t* leaf_parent, uint32_t* root, cudaStream_t st);
// Every internal node's child record (dpc_device.cuh: the children's
// indices, their largest order keys and, with `boxes`, their bounding boxes
// over all dp coordinates) into nrec, kRecWordsMax words per node at most;
// the boxes depend only on the points, so once per binning suffices.
void launch_tree_maxkey(const unsigned long long* skey, const float* spts, int dp, uint32_t n,
                        Node* nodes, const uint32_t* leaf_parent, uint32_t* visit, float* nrec,
                        bool boxes, cudaStream_t st);

// Work layouts of the density and near-dependent kernels:
//   union    a warp owns 32 consecutive sorted points (one query per lane) and
//            streams the union of their blocks through shared memory, every
//            candidate a broadcast read (block.cuh)
//   segment  the 32 points are split into segments of equal cell; the block's
//            candidates are spread over the lanes (in registers) and the
//            segment's queries are taken one at a time, one warp reduction each
//   tree     (near phase only) no block scan: every query goes to the tree
//            search of the far phase
//   tensor   (density, 5-8 dimensions, float32 filter) the distance tiles on the
//            tensor cores (tc_density.cu); other cases fall back to segment
//   pairs    (density only) the segment layout counting every unordered pair
//            once, for both of its points (density.cu, k_density_pairs)
// seg_cells (segment layouts): a segment may span several consecutive cells
// while their bounding box grown by R holds at most seg_cells cells (0: one
// cell per segment)
//   cell     one warp per occupied cell: the block's points staged in shared
//            memory, every lane one query (or a share of one query's
//            candidates for cells below 32 points) against all of them
//            (cell_tile.cu)
enum { kLayoutUnion = 1, kLayoutSegment = 2, kLayoutTree = 3, kLayoutTensor = 4, kLayoutPairs = 5,
       kLayoutCell = 6 };

// ---- density (density.cu) -------------------------------------------------------
// rho of every point for one cutoff (cuts: [ninst]); rho_out is indexed by
// output index (sid)
void launch_density(int dp, int g, bool fp64, int layout, const float* spts,
                    const unsigned long long* scode, const uint32_t* sid, const ClassView& cv,
                    const CutGeom* cuts, HashInfo* hi, const unsigned long long* hkeys,
                    const uint2* hvals, uint2* pieces, int32_t* rho_out,
                    unsigned long long* skey, Counters* ctr, cudaStream_t st,
                    int seg_cells = 0);
// the tensor-core form of the density step (dp = 8, float32 filter only)
// (pieces: scratch for the piece list, at least N / 128 + occupied cells entries)
void launch_density_tc(int g, const float* spts, const uint32_t* sid, const ClassView& cv,
                       const CutGeom* cuts, HashInfo* hi, const unsigned long long* hkeys,
                       const uint2* hvals, uint2* pieces, int32_t* rho_out,
                       unsigned long long* skey, Counters* ctr, cudaStream_t st);
// the cell layout of the density step (cell_tile.cu)
void launch_density_cell(int dp, int g, bool fp64, const float* spts,
                         const unsigned long long* scode, const uint32_t* sid, const ClassView& cv,
                         const CutGeom* cuts, const HashInfo* hi, const unsigned long long* hkeys,
                         const uint2* hvals, int32_t* rho_out, unsigned long long* skey,
                         Counters* ctr, cudaStream_t st);
// order keys of sorted points from densities given by output index
void launch_keys_from_rho(const int32_t* rho, const uint32_t* sid, uint32_t n,
                          unsigned long long* skey, cudaStream_t st);

// ---- dependent points (dependent.cu) ----------------------------------------------
struct FarQueue {
  uint32_t* pos;   // sorted position of each queued query
  float* s1;       // best float32 distance found by the near phase (FP32 mode)
  double* s1d;     // best binary64 distance found by the near phase (FP64 mode)
  uint32_t* pos2;  // the same for the queries passed to the far phase's second round
  float* s1_2;
  double* s1d2;
};
// lambda and delta are indexed by output index; lambda values are
// instance-local ids
void launch_dep_near(int dp, int g, bool fp64, int layout, const float* spts,
                     const unsigned long long* scode, const unsigned long long* skey,
                     const ClassView& cv, int32_t rho_skip, const void* pts, int dtype,
                     const CutGeom* cuts, const HashInfo* hi, const unsigned long long* hkeys,
                     const uint2* hvals, int32_t* lambda, double* delta, FarQueue q, Counters* ctr,
                     cudaStream_t st,
                     int seg_cells = 0);
// the cell layout of the near phase (cell_tile.cu)
void launch_dep_near_cell(int dp, int g, bool fp64, const float* spts,
                          const unsigned long long* scode, const unsigned long long* skey,
                          const ClassView& cv, int32_t rho_skip, const void* pts, int dtype,
                          const CutGeom* cuts, const HashInfo* hi,
                          const unsigned long long* hkeys, const uint2* hvals, int32_t* lambda,
                          double* delta, FarQueue q, Counters* ctr, cudaStream_t st);
// the tensor-core form of the near phase (dp = 8, float32 filter only;
// pieces: scratch as for launch_density_tc)
void launch_dep_near_tc(int g, const float* spts, const uint32_t* sid,
                        const unsigned long long* skey, const ClassView& cv, int32_t rho_skip,
                        const void* pts, int dtype, const CutGeom* cuts, HashInfo* hi,
                        const unsigned long long* hkeys, const uint2* hvals, uint2* pieces,
                        int32_t* lambda, double* delta, FarQueue q, Counters* ctr,
                        cudaStream_t st);
void launch_dep_far(int dp, bool fp64, const float* spts, const unsigned long long* scode,
                    const unsigned long long* skey, const ClassView& cv, const CutGeom* cuts,
                    const Node* nodes, const float* nbox, const uint32_t* root, FarQueue q,
                    int32_t* lambda, double* delta, Counters* ctr, cudaStream_t st);

// ---- decision graph (decision.cu) -------------------------------------------------
// top-k by gamma = rho * delta and the (rho, delta) histogram of every instance
// of the class (rho, delta indexed by output index; top/gamma [n_inst][k] and
// hist [n_inst][rho_bins][delta_bins] by batch row, InstDev::row)
void launch_decision(const int32_t* rho, const double* delta, const ClassView& cv, int k,
                     int32_t* top, double* gamma, int rho_bins, int delta_bins, double delta_lo,
                     unsigned long long* hist, void* scratch, cudaStream_t st);
// device scratch launch_decision needs for a class of ninst instances
size_t decision_scratch_bytes(uint32_t ninst, int k);
// ---- priority range search (range.cu) -------------------------------------------
struct PrangeArgs {
  uint32_t nq;              // queries
  int32_t n_inst;           // instances of the batch
  const int32_t* q_inst;    // [nq] batch row of each query (device)
  const double* q_box;      // [nq][2][kMaxDim] lo then hi (device)
  const int32_t* q_rho;     // [nq] thresholds (device)
  const int32_t* rowmap;    // [n_inst] class-local index or -1; null: one_row only
  int32_t one_row;          // the batch row of a single-instance class
  long long* count;         // [nq] matches (device output)
  int stack_cap;            // shared stack entries per warp (0: all); smaller
                            //   values send more subtrees to the per-lane walk
};
void launch_prange_init(const PrangeArgs& a, int32_t* ids, int max_out, int* status,
                        cudaStream_t st);
// one class: count (fill = false: cnt[q] for the class's queries, 0 for the
// others, and count[q]) or fill (keys (q << 31 | id) at off[q]..)
void launch_prange(int dp, bool fill, const float* spts, const uint32_t* sid,
                   const unsigned long long* skey, const ClassView& cv, const Node* nodes,
                   const float* nbox, const uint32_t* roots, const PrangeArgs& a, uint32_t* cnt,
                   const unsigned long long* off, unsigned long long* keys, int* status,
                   cudaStream_t st);
void launch_prange_scan(const uint32_t* cnt, uint32_t nq, unsigned long long* off, cudaStream_t st);
void launch_prange_scatter(const unsigned long long* keys, uint64_t total,
                           const unsigned long long* off, uint32_t nq, int max_out, int32_t* ids,
                           int* status, cudaStream_t st);

int decision_max_topk();
// padding of every top-k row (-1, NaN) and zero histograms for n_inst rows
void launch_decision_init(int n_inst, int k, int32_t* top, double* gamma, int rho_bins,
                          int delta_bins, unsigned long long* hist, cudaStream_t st);

// ---- labels (labels.cu) -------------------------------------------------------------
int label_rounds(uint32_t n);
// Labels of every point of the class for one cutoff (arrays indexed by output
// index); params: [ninst] on the device, or null for a single instance (`one`);
// nmax: the largest instance; flags needs label_rounds(nmax) + 1 ints.
void launch_labels(const int32_t* rho, const int32_t* lambda, const double* delta,
                   const ClassView& cv, uint32_t nmax, const LabelParams* params,
                   LabelParams one, int32_t* label, int32_t* flags, cudaStream_t st);

}  // namespace dpc
