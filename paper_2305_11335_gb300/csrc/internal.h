// internal.h -- host-side launchers of the library's kernels (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpc_device.cuh"

namespace dpc {

// Kernels enqueued by the current call (the entry points hold the library
// lock while enqueueing, so a plain counter suffices).
extern long long g_kernel_launches;
inline void count_launches(int k) { g_kernel_launches += k; }

// Host-computed constants of one cutoff (the [host] fields of CutGeom).
struct CutHost {
  double dc, dc2;
  float t_in, t_out, band_mul, band_add;
};
CutHost make_cut_host(double d_cut, int dp);

// ---- binning (binning.cu) ---------------------------------------------------
void launch_geom_init(GridGeom* geom, int* status, int g, cudaStream_t st);
void launch_bbox(const void* pts, int dtype, uint32_t n, int d, int g, GridGeom* geom,
                 cudaStream_t st);
void launch_setup(GridGeom* geom, CutGeom* cuts, const CutHost* host_cuts, int ncut,
                  cudaStream_t st);
void launch_codes(const void* pts, int dtype, uint32_t n, int d, const GridGeom* geom,
                  unsigned long long* codes, uint32_t* ids, cudaStream_t st);
void launch_gather(const void* pts, int dtype, uint32_t n, int d, int dp, const GridGeom* geom,
                   const unsigned long long* codes_a, const unsigned long long* codes_b,
                   const uint32_t* ids_a, const uint32_t* ids_b, float* spts,
                   unsigned long long* scode, uint32_t* sid, cudaStream_t st);
void launch_cells(const unsigned long long* scode, uint32_t n, const GridGeom* geom, CutGeom* cut,
                  unsigned long long* hkeys, uint2* hvals, uint32_t hcap, cudaStream_t st);

// ---- radix sort (sort.cu) ------------------------------------------------------
size_t sort_hist_words(uint32_t n);
// Sorts (codes_a, ids_a) by code, LSD over the device-side pass count
// geom->npass; the result lands in the _a buffers if npass is even, else _b.
void launch_sort(unsigned long long* codes_a, unsigned long long* codes_b, uint32_t* ids_a,
                 uint32_t* ids_b, uint32_t n, const GridGeom* geom, uint32_t* hist,
                 cudaStream_t st);

// ---- radix tree (tree.cu) ------------------------------------------------------
void launch_tree_build(const unsigned long long* scode, uint32_t n, const GridGeom* geom,
                       Node* nodes, uint32_t* leaf_parent, cudaStream_t st);
// Largest order key of every subtree; with `boxes`, also every node's
// bounding box over all dp coordinates into nbox ([lo(dp) | hi(dp)] floats per
// node; the box depends only on the points, so once per binning suffices).
void launch_tree_maxkey(const unsigned long long* skey, const float* spts, int dp, uint32_t n,
                        Node* nodes, const uint32_t* leaf_parent, uint32_t* visit, float* nbox,
                        bool boxes, cudaStream_t st);

// ---- density (density.cu) -------------------------------------------------------
void launch_density(int dp, int g, bool fp64, const float* spts, const unsigned long long* scode,
                    const uint32_t* sid, uint32_t n, const GridGeom* geom, const CutGeom* cut,
                    const unsigned long long* hkeys, const uint2* hvals, int32_t* rho_out,
                    unsigned long long* skey, Counters* ctr, cudaStream_t st);
// order keys of sorted points from densities given in original order
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
void launch_dep_near(int dp, int g, bool fp64, const float* spts, const unsigned long long* scode,
                     const unsigned long long* skey, uint32_t n, int32_t rho_skip, const void* pts,
                     int dtype, int d, const GridGeom* geom, const CutGeom* cut, const unsigned long long* hkeys,
                     const uint2* hvals, int32_t* lambda, double* delta, FarQueue q,
                     Counters* ctr, cudaStream_t st);
void launch_dep_far(int dp, bool fp64, const float* spts, const unsigned long long* skey,
                    uint32_t n, const GridGeom* geom, const CutGeom* cut, const Node* nodes,
                    const float* nbox, FarQueue q, int32_t* lambda, double* delta, Counters* ctr,
                    uint32_t qcap, cudaStream_t st);

// ---- labels (labels.cu) -------------------------------------------------------------
int label_rounds(uint32_t n);
void launch_labels(const int32_t* rho, const int32_t* lambda, const double* delta, uint32_t n,
                   int32_t rho_noise, int32_t rho_min, double delta_min, int32_t* label,
                   int32_t* flags, GridGeom* geom, cudaStream_t st);

}  // namespace dpc
