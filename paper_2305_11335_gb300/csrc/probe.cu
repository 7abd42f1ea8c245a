// probe.cu -- measured arithmetic peaks for the roofline of the search kernels.
//
// The distance kernels are bound by float32 issue (one fused multiply-add per
// coordinate and candidate) and their binary64 recheck by the FP64 pipe, so
// their roofline denominators are the chip's FFMA and DFMA rates, measured
// here at the clocks the GPU runs at: every thread runs kChains independent
// multiply-add chains for `iters` steps (enough independent work to fill the
// pipes), on a grid of a few CTAs per SM, timed with CUDA events.
#include <algorithm>
#include <vector>

#include "../../include/dpc.h"
#include "internal.h"

namespace dpc {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_loop(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int iters, cudaStream_t st, double* flops_per_s) {
  const unsigned grid = sm_count() * 4u;
  T* out = nullptr;
  if (!dev_alloc((void**)&out, sizeof(T) * grid * kProbeThreads)) return DPC_ERR_OOM;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // b and c keep the chains bounded (|a| stays near c / (1 - b))
  const T mul = (T)0.999, add = (T)0.001;
  k_fma_loop<T><<<grid, kProbeThreads, 0, st>>>(out, iters, mul, add);  // warm-up
  std::vector<float> ms;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(a, st);
    k_fma_loop<T><<<grid, kProbeThreads, 0, st>>>(out, iters, mul, add);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    ms.push_back(t);
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (err != cudaSuccess) return DPC_ERR_CUDA;
  std::sort(ms.begin(), ms.end());
  const double flops = 2.0 * kChains * (double)iters * grid * kProbeThreads;
  *flops_per_s = flops / (ms[ms.size() / 2] * 1e-3);
  return DPC_OK;
}

}  // namespace
}  // namespace dpc

extern "C" int dpc_probe_peak(int kind, double* flops_per_s, void* stream) {
  if (!flops_per_s || (kind != 0 && kind != 1)) return DPC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return kind == 0 ? dpc::probe<float>(1 << 17, st, flops_per_s)
                   : dpc::probe<double>(1 << 12, st, flops_per_s);
}
