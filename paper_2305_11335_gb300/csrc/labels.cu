// labels.cu -- noise, centers and cluster labels (Definitions 4-5 and the
// assignment rule after them).
//
// The paper links every non-center point to its dependent point with a
// concurrent union-find (Algorithm 3).  The dependent pointers already form a
// forest with one parent edge per point, so the components are found here by
// pointer jumping instead: each round makes every pointer jump several times
// towards its root (see k_label_jump for the rate).  Rounds are launched a
// fixed number of times (label_rounds: enough for any forest of n points);
// a round after one in which every pointer reached its root returns at once,
// so the launch sequence does not depend on the data.  A pointer still short
// of a root after the last round means the input was not a forest, recorded
// as kStatusCycle.
#include "internal.h"

namespace dpc {

namespace {

constexpr int kThreads = 256;

// Every point of the class once: f(inst, output index, instance).
template <typename F>
__device__ __forceinline__ void for_class_points(const ClassView& cv, F f) {
  if (!cv.chunk_inst) {  // one instance: positions 0 .. N-1
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < cv.N; p += gridDim.x * blockDim.x)
      f(0u, (int32_t)(cv.one.out + p), cv.one);
    return;
  }
  const uint64_t total = (uint64_t)cv.nchunk * 32u;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t inst, p0, end;
    cv.chunk((uint32_t)(e >> 5), inst, p0, end);
    const uint32_t p = p0 + (uint32_t)(e & 31u);
    if (p >= end) continue;
    const InstDev I = cv.instance(inst);
    f(inst, (int32_t)(I.out + (p - I.start)), I);
  }
}

// par[i] = -1 (noise), i (center) or lambda_i (follows its dependent point),
// all as output indices.
__global__ void k_label_init(const int32_t* __restrict__ rho, const int32_t* __restrict__ lambda,
                             const double* __restrict__ delta, ClassView cv,
                             const LabelParams* __restrict__ params, LabelParams one,
                             int32_t* __restrict__ par, int32_t* __restrict__ flags) {
  for_class_points(cv, [&](uint32_t inst, int32_t i, const InstDev& I) {
    const LabelParams P = params ? params[inst] : one;
    const int32_t r = rho[i];
    const int32_t l = lambda[i];
    int32_t v;
    if (r < P.rho_noise) v = -1;                                             // Definition 4
    else if (l < 0 || (r >= P.rho_min && delta[i] >= P.delta_min)) v = i;    // Definition 5
    else v = (l < (int32_t)I.n) ? (int32_t)(I.out + (uint32_t)l) : -1;
    par[i] = v;
  });
  if (blockIdx.x == 0 && threadIdx.x == 0) flags[0] = 1;  // round 0 always runs
}

// Round r (1-based): up to kJumps times, par[i] <- par[par[i]].  Pointers only
// ever move towards the root, so concurrent updates by other threads are
// harmless.  If every pointer covered at least L steps before a round, the
// first jump covers 2L and each further one at least L more, so a round
// multiplies the covered distance by at least kJumps + 1.  A pointer that
// reached a root (a center, which points to itself, or noise) is final; the
// next round runs only if some pointer has not (flags[r]).  Only thread i
// writes par[i], and never i itself: a walk that comes back to its own point
// is on a cycle, and writing it as its own parent would make a root of it,
// so the points of a cycle (and those leading into it) never reach a root
// and the flag of the last round reports it.
constexpr int kJumps = 32;
__global__ void k_label_jump(int32_t* par, ClassView cv, int32_t* flags, int r) {
  if (flags[r - 1] == 0) return;  // every pointer reached its root before
  int open = 0;
  for_class_points(cv, [&](uint32_t, int32_t i, const InstDev&) {
    int32_t p = par[i];
    if (p < 0 || p == i) return;
    const int32_t p0 = p;
    bool root = false;
#pragma unroll 1
    for (int j = 0; j < kJumps; ++j) {
      const int32_t pp = par[p];
      if (pp == p || pp < 0) {
        if (pp < 0) p = pp;
        root = true;
        break;
      }
      p = pp;
      if (p == i) break;  // back at itself: a cycle, never written as a root
    }
    if (p != p0 && p != i) par[i] = p;
    if (!root) open = 1;
  });
  if (__syncthreads_or(open) && threadIdx.x == 0) flags[r] = 1;
}

// Output indices of the centers back to instance-local ids.
__global__ void k_label_local(int32_t* par, ClassView cv) {
  for_class_points(cv, [&](uint32_t, int32_t i, const InstDev& I) {
    const int32_t v = par[i];
    par[i] = v < 0 ? -1 : (int32_t)((uint32_t)v - (uint32_t)I.out);
  });
}

__global__ void k_label_check(const int32_t* __restrict__ flags, int last, ClassGeom* cls) {
  if (flags[last]) set_status(cls->status, kStatusCycle);
}

inline unsigned grid_for(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > sm_count() * 16u) b = sm_count() * 16u;
  return (unsigned)b;
}

}  // namespace

// Rounds until every chain (at most n - 1 long) has reached its root (the
// smallest r with (kJumps + 1)^r >= n), one in which a pointer that landed on
// its root with its last jump sees it, and one more whose flag the check
// reads (0 for a forest): r + 2.
int label_rounds(uint32_t n) {
  int r = 0;
  unsigned long long reach = 1;
  while (reach < (unsigned long long)n) {
    reach *= (unsigned long long)(kJumps + 1);
    ++r;
  }
  return r + 2;
}

// `label` doubles as the pointer array; `flags` needs label_rounds(nmax) + 1 ints.
void launch_labels(const int32_t* rho, const int32_t* lambda, const double* delta,
                   const ClassView& cv, uint32_t nmax, const LabelParams* params,
                   LabelParams one, int32_t* label, int32_t* flags, cudaStream_t st) {
  if (cv.N == 0) return;
  const int rounds = label_rounds(nmax);
  cudaMemsetAsync(flags, 0, sizeof(int32_t) * (rounds + 1), st);
  const unsigned grid = grid_for((uint64_t)cv.nchunk * 32u);
  k_label_init<<<grid, kThreads, 0, st>>>(rho, lambda, delta, cv, params, one, label, flags);
  for (int r = 1; r <= rounds; ++r) k_label_jump<<<grid, kThreads, 0, st>>>(label, cv, flags, r);
  k_label_local<<<grid, kThreads, 0, st>>>(label, cv);
  k_label_check<<<1, 1, 0, st>>>(flags, rounds, cv.cls);
  count_launches(rounds + 3);
}

}  // namespace dpc
