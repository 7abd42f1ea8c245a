// static_density.cu -- dpc_density for one point set without any device
// allocation: every scratch buffer lives in one file-scope __device__ array.
//
// For callers that must not allocate device memory: hosts whose device memory
// is handed out by their own allocator or budget, and latency-critical paths
// (cudaMalloc and cudaFree may synchronize the device).  The price is a fixed
// maximum size and a single shared scratch area (see dpc.h).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/dpc.h"
#include "internal.h"

namespace dpc {
namespace {

constexpr uint64_t kStaticN = DPC_STATIC_MAX_POINTS;
constexpr size_t kA = 256;

constexpr size_t al(size_t x) { return (x + kA - 1) / kA * kA; }
constexpr uint32_t pow2_at_least(uint64_t x) {
  uint64_t t = 16;
  while (t < x) t <<= 1;
  return (uint32_t)t;
}
constexpr uint32_t kStaticHash = pow2_at_least(2 * kStaticN);

// Layout of the scratch array (byte offsets).
constexpr size_t kOffGeom = 0;
constexpr size_t kOffCut = kOffGeom + al(sizeof(GridGeom));
constexpr size_t kOffCls = kOffCut + al(sizeof(CutGeom));
constexpr size_t kOffHash = kOffCls + al(sizeof(ClassGeom));
constexpr size_t kOffCtr = kOffHash + al(sizeof(HashInfo));
constexpr size_t kOffStatus = kOffCtr + al(sizeof(Counters));
constexpr size_t kOffCodesA = kOffStatus + al(sizeof(int));
constexpr size_t kOffCodesB = kOffCodesA + al(8 * kStaticN);
constexpr size_t kOffIdsA = kOffCodesB + al(8 * kStaticN);
constexpr size_t kOffIdsB = kOffIdsA + al(4 * kStaticN);
constexpr size_t kOffHist = kOffIdsB + al(4 * kStaticN);
constexpr size_t kOffSpts = kOffHist + al(4 * sort_hist_words_for(kStaticN));
constexpr size_t kOffScode = kOffSpts + al(4 * 8 * kStaticN);
constexpr size_t kOffSid = kOffScode + al(8 * kStaticN);
constexpr size_t kOffSkey = kOffSid + al(4 * kStaticN);
constexpr size_t kOffHkeys = kOffSkey + al(8 * kStaticN);
constexpr size_t kOffHvals = kOffHkeys + al(8 * (size_t)kStaticHash);
constexpr size_t kStaticBytes = kOffHvals + al(8 * (size_t)kStaticHash);

// The scratch area.  In host code this name is only a handle; its device
// address comes from cudaGetSymbolAddress (once per device, below).
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];
// the sort's scratch for the largest accepted set fits its region
static_assert(kOffSpts - kOffHist >= 4 * sort_hist_words_for(kStaticN), "sort scratch region");

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch area on the current device, looked up on
// the first call for that device.
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return DPC_OK;
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" int dpc_density_static(const void* pts, int dtype, int64_t n, int32_t d, double d_cut,
                                  int32_t* rho, uint32_t flags, void* stream) {
  const uint32_t prec = flags & DPC_PREC_MASK;
  if (prec != DPC_PREC_FP64 && prec != DPC_PREC_FP32_CERT) return DPC_ERR_UNSUPPORTED;
  if (flags & ~(DPC_PREC_MASK | DPC_FLAG_SYNC_CHECK)) return DPC_ERR_ARG;
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (d < 1 || d > kMaxDim || n < 0 || !(d_cut >= 0.0) || d_cut > 1.7e308) return DPC_ERR_ARG;
  if ((uint64_t)n > kStaticN) return DPC_ERR_OVERFLOW;
  if (n > 0 && (!pts || !rho)) return DPC_ERR_ARG;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  if (n == 0) return DPC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_static_mu);

  GridGeom* geom = (GridGeom*)(base + kOffGeom);
  CutGeom* cut = (CutGeom*)(base + kOffCut);
  ClassGeom* cls = (ClassGeom*)(base + kOffCls);
  HashInfo* hinfo = (HashInfo*)(base + kOffHash);
  Counters* ctr = (Counters*)(base + kOffCtr);
  int* status = (int*)(base + kOffStatus);
  unsigned long long* codes_a = (unsigned long long*)(base + kOffCodesA);
  unsigned long long* codes_b = (unsigned long long*)(base + kOffCodesB);
  uint32_t* ids_a = (uint32_t*)(base + kOffIdsA);
  uint32_t* ids_b = (uint32_t*)(base + kOffIdsB);
  uint32_t* hist = (uint32_t*)(base + kOffHist);
  float* spts = (float*)(base + kOffSpts);
  unsigned long long* scode = (unsigned long long*)(base + kOffScode);
  uint32_t* sid = (uint32_t*)(base + kOffSid);
  unsigned long long* skey = (unsigned long long*)(base + kOffSkey);
  unsigned long long* hkeys = (unsigned long long*)(base + kOffHkeys);
  uint2* hvals = (uint2*)(base + kOffHvals);

  const uint32_t nn = (uint32_t)n;
  const int g = grid_dims(d);
  const int dp = d <= 2 ? 2 : (d <= 4 ? 4 : 8);
  const CutHost ch = make_cut_host(d_cut, dp);
  // the previous call's contents are still there: zero the words that
  // accumulate (status, counters); every other buffer is fully rewritten
  cudaMemsetAsync(status, 0, sizeof(int), st);
  cudaMemsetAsync(ctr, 0, sizeof(Counters), st);
  // one instance: a class without instance or chunk tables
  ClassView cv;
  memset(&cv, 0, sizeof(cv));
  cv.N = nn;
  cv.ninst = 1;
  cv.nchunk = (nn + 31) / 32;
  cv.one.n = nn;
  cv.one.d = d;
  cv.geom = geom;
  cv.cls = cls;
  // one instance: no instance bits, and g * B <= 63 keeps every cell code
  // below 2^63 (the allocating path's rule with ib = 0)
  launch_class_init(cv, g, 0, std::min(kMaxBits, 63 / g), status, st);
  launch_bbox(pts, dtype, cv, g, st);
  launch_setup(cv, cut, 1, nullptr, &ch, st);
  launch_codes(pts, dtype, cv, g, codes_a, ids_a, st);
  launch_sort(codes_a, codes_b, ids_a, ids_b, nn, cls, hist, st);
  launch_gather(pts, dtype, cv, dp, codes_a, codes_b, ids_a, ids_b, spts, scode, sid, st);
  launch_cells(scode, cv, g, cut, hinfo, hkeys, hvals, kStaticHash, st);
  launch_density(dp, g, prec == DPC_PREC_FP64, g >= 2 ? kLayoutSegment : kLayoutUnion, spts, scode,
                 sid, cv, cut, hinfo, hkeys, hvals, nullptr, rho,
                 skey, ctr, st);
  if (cudaGetLastError() != cudaSuccess) return DPC_ERR_CUDA;
  if (flags & DPC_FLAG_SYNC_CHECK) {
    int s = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(&s, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    if (s & kStatusBadCoord) return DPC_ERR_DATA;
    if (s) return DPC_ERR_CUDA;
  }
  return DPC_OK;
}
