// labels.cu -- noise, centers and cluster labels (Definitions 4-5 and the
// assignment rule after them).
//
// The paper links every non-center point to its dependent point with a
// concurrent union-find (Algorithm 3).  The dependent pointers already form a
// forest with one parent edge per point, so the components are found here by
// pointer jumping instead: each round makes every pointer jump several times
// towards its root (see k_label_jump for the rate).  Rounds are launched a
// fixed number of times (label_rounds: enough for any forest of n points);
// a round that sees no change in the previous one returns at once, so the
// launch sequence does not depend on the data.  A pointer still moving after
// the last round means the input was not a forest, recorded as kStatusCycle.
#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 256;

// par[i] = -1 (noise), i (center) or lambda_i (follows its dependent point).
__global__ void k_label_init(const int32_t* __restrict__ rho, const int32_t* __restrict__ lambda,
                             const double* __restrict__ delta, uint32_t n, int32_t rho_noise,
                             int32_t rho_min, double delta_min, int32_t* __restrict__ par,
                             int32_t* __restrict__ flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t r = rho[i];
    const int32_t l = lambda[i];
    int32_t v;
    if (r < rho_noise) v = -1;                                        // Definition 4
    else if (l < 0 || (r >= rho_min && delta[i] >= delta_min)) v = (int32_t)i;  // Definition 5
    else v = (l < (int32_t)n) ? l : -1;
    par[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) flags[0] = 1;  // round 0 always runs
}

// Round r (1-based): up to kJumps times, par[i] <- par[par[i]].  Pointers only
// ever move towards the root, so concurrent updates by other threads are
// harmless.  If every pointer covered at least L steps before a round, the
// first jump covers 2L and each further one at least L more, so a round
// multiplies the covered distance by at least kJumps + 1.
constexpr int kJumps = 8;
__global__ void k_label_jump(int32_t* par, uint32_t n, int32_t* flags, int r) {
  if (flags[r - 1] == 0) return;  // the previous round changed nothing
  int changed = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t p = par[i];
    if (p < 0 || p == (int32_t)i) continue;
    int32_t p0 = p;
#pragma unroll 1
    for (int j = 0; j < kJumps; ++j) {
      const int32_t pp = par[p];
      if (pp == p || pp < 0) {
        if (pp < 0) p = pp;
        break;
      }
      p = pp;
    }
    if (p != p0) {
      par[i] = p;
      changed = 1;
    }
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) flags[r] = 1;
}

__global__ void k_label_check(const int32_t* __restrict__ flags, int last, GridGeom* geom) {
  if (flags[last]) set_status(geom->status, kStatusCycle);
}

inline unsigned grid_for(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152u * 16u) b = 152u * 16u;
  return (unsigned)b;
}

}  // namespace

// Rounds until every chain (at most n - 1 long) has reached its root, plus
// one that sees no change: the smallest r with (kJumps + 1)^r >= n, plus 2.
int label_rounds(uint32_t n) {
  int r = 0;
  unsigned long long reach = 1;
  while (reach < (unsigned long long)n) {
    reach *= (unsigned long long)(kJumps + 1);
    ++r;
  }
  return r + 2;
}

// `label` doubles as the pointer array; `flags` needs label_rounds(n) + 1 ints.
void launch_labels(const int32_t* rho, const int32_t* lambda, const double* delta, uint32_t n,
                   int32_t rho_noise, int32_t rho_min, double delta_min, int32_t* label,
                   int32_t* flags, GridGeom* geom, cudaStream_t st) {
  if (n == 0) return;
  const int rounds = label_rounds(n);
  cudaMemsetAsync(flags, 0, sizeof(int32_t) * (rounds + 1), st);
  const unsigned grid = grid_for(n);
  k_label_init<<<grid, kThreads, 0, st>>>(rho, lambda, delta, n, rho_noise, rho_min, delta_min,
                                          label, flags);
  for (int r = 1; r <= rounds; ++r) k_label_jump<<<grid, kThreads, 0, st>>>(label, n, flags, r);
  k_label_check<<<1, 1, 0, st>>>(flags, rounds, geom);
  count_launches(rounds + 2);
}

}  // namespace dpc
