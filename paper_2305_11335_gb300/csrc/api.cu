// api.cu -- the C ABI (include/dpc.h): argument checks, the per-(device,
// stream) workspace, and the order in which the kernels run.
//
// Pipeline of one instance (all on the caller's stream, no host sync):
//   binning   bbox -> grid setup -> Morton codes -> radix sort -> gather
//   tree      radix tree over the sorted codes (dependent points only)
//   per cutoff
//     cells     occupied level-k cells -> hash
//     density   rho (Definition 1) + order keys
//     dependent maxkeys of the tree -> near phase -> far phase (Definitions 2-3)
//     labels    pointer jumping (Definitions 4-5)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/dpc.h"
#include "internal.h"

namespace dpc {

long long g_kernel_launches = 0;

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

inline uint32_t next_pow2(uint64_t x) {
  uint64_t t = 16;
  while (t < x) t <<= 1;
  return (uint32_t)t;
}

struct Workspace {
  int device = -1;
  cudaStream_t stream = nullptr;
  uint64_t cap_n = 0;     // points per instance the buffers hold
  int cap_ncut = 0;
  void* base = nullptr;   // one allocation, carved below
  size_t bytes = 0;

  GridGeom* geom = nullptr;
  CutGeom* cuts = nullptr;
  Counters* ctr = nullptr;
  int* status = nullptr;
  int32_t* flags = nullptr;
  unsigned long long *codes_a = nullptr, *codes_b = nullptr;
  uint32_t *ids_a = nullptr, *ids_b = nullptr;
  uint32_t* hist = nullptr;
  float* spts = nullptr;
  unsigned long long* scode = nullptr;
  uint32_t* sid = nullptr;
  unsigned long long* skey = nullptr;
  unsigned long long* hkeys = nullptr;
  uint2* hvals = nullptr;
  uint32_t hcap = 0;
  Node* nodes = nullptr;
  float* nbox = nullptr;    // per-node bounding boxes, [lo(dp) | hi(dp)]
  bool boxes_ready = false; // nbox matches the current binning
  uint32_t* leaf_parent = nullptr;
  uint32_t* visit = nullptr;
  uint32_t* qpos = nullptr;
  float* qs1 = nullptr;
  double* qs1d = nullptr;
  uint32_t* qpos2 = nullptr;
  float* qs1_2 = nullptr;
  double* qs1d2 = nullptr;

  // host-buffer entry point staging
  void* io = nullptr;
  size_t io_bytes = 0;

  int last_level = 0;     // for dpc_get_stats
  int last_ncut_used = 0;
  long long launches_last = 0;

  // phase timing (DPC_FLAG_PHASE_TIMES)
  struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<PhaseRec> recs;

  cudaEvent_t take_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }

  void begin_call(uint32_t flags) {
    timing = (flags & DPC_FLAG_PHASE_TIMES) != 0;
    recs.clear();
    ev_used = 0;
    g_kernel_launches = 0;
  }
  void end_call() { launches_last = g_kernel_launches; }

  void release() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    ev_used = 0;
    recs.clear();
    if (base) cudaFree(base);
    if (io) cudaFree(io);
    base = nullptr;
    io = nullptr;
    bytes = io_bytes = 0;
    cap_n = 0;
    cap_ncut = 0;
  }

  int reserve(uint64_t n, int ncut) {
    if (n <= cap_n && ncut <= cap_ncut && base) return DPC_OK;
    uint64_t want_n = n > cap_n ? n : cap_n;
    int want_c = ncut > cap_ncut ? ncut : cap_ncut;
    if (want_n < 1024) want_n = 1024;
    if (want_c < 8) want_c = 8;
    if (base) {
      cudaStreamSynchronize(stream);
      cudaFree(base);
      base = nullptr;
    }
    const uint64_t N = want_n;
    const uint32_t hc = next_pow2(2 * N);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align_up(b); return o; };
    const size_t o_geom = take(sizeof(GridGeom));
    const size_t o_cuts = take(sizeof(CutGeom) * want_c);
    const size_t o_ctr = take(sizeof(Counters));
    const size_t o_status = take(sizeof(int));
    const size_t o_flags = take(sizeof(int32_t) * 80);
    const size_t o_ca = take(8 * N), o_cb = take(8 * N);
    const size_t o_ia = take(4 * N), o_ib = take(4 * N);
    const size_t o_hist = take(4 * sort_hist_words((uint32_t)N));
    const size_t o_spts = take(4 * 8 * N);
    const size_t o_scode = take(8 * N);
    const size_t o_sid = take(4 * N);
    const size_t o_skey = take(8 * N);
    const size_t o_hk = take(8 * (size_t)hc), o_hv = take(8 * (size_t)hc);
    const size_t o_nodes = take(sizeof(Node) * N);
    const size_t o_nbox = take(4 * 16 * N);
    const size_t o_lp = take(4 * N), o_visit = take(4 * N);
    const size_t o_qpos = take(4 * N), o_qs1 = take(4 * N), o_qs1d = take(8 * N);
    const size_t o_qpos2 = take(4 * N), o_qs1_2 = take(4 * N), o_qs1d2 = take(8 * N);
    void* p = nullptr;
    if (cudaMalloc(&p, off) != cudaSuccess) {
      cudaGetLastError();
      cap_n = 0;
      return DPC_ERR_OOM;
    }
    base = p;
    bytes = off;
    char* b = (char*)p;
    geom = (GridGeom*)(b + o_geom);
    cuts = (CutGeom*)(b + o_cuts);
    ctr = (Counters*)(b + o_ctr);
    status = (int*)(b + o_status);
    flags = (int32_t*)(b + o_flags);
    codes_a = (unsigned long long*)(b + o_ca);
    codes_b = (unsigned long long*)(b + o_cb);
    ids_a = (uint32_t*)(b + o_ia);
    ids_b = (uint32_t*)(b + o_ib);
    hist = (uint32_t*)(b + o_hist);
    spts = (float*)(b + o_spts);
    scode = (unsigned long long*)(b + o_scode);
    sid = (uint32_t*)(b + o_sid);
    skey = (unsigned long long*)(b + o_skey);
    hkeys = (unsigned long long*)(b + o_hk);
    hvals = (uint2*)(b + o_hv);
    hcap = hc;
    nodes = (Node*)(b + o_nodes);
    nbox = (float*)(b + o_nbox);
    leaf_parent = (uint32_t*)(b + o_lp);
    visit = (uint32_t*)(b + o_visit);
    qpos = (uint32_t*)(b + o_qpos);
    qs1 = (float*)(b + o_qs1);
    qs1d = (double*)(b + o_qs1d);
    qpos2 = (uint32_t*)(b + o_qpos2);
    qs1_2 = (float*)(b + o_qs1_2);
    qs1d2 = (double*)(b + o_qs1d2);
    cap_n = N;
    cap_ncut = want_c;
    cudaMemsetAsync(status, 0, sizeof(int), stream);
    cudaMemsetAsync(ctr, 0, sizeof(Counters), stream);
    return DPC_OK;
  }

  int reserve_io(size_t b) {
    if (b <= io_bytes && io) return DPC_OK;
    if (io) {
      cudaStreamSynchronize(stream);
      cudaFree(io);
      io = nullptr;
    }
    if (cudaMalloc(&io, b) != cudaSuccess) {
      cudaGetLastError();
      io_bytes = 0;
      return DPC_ERR_OOM;
    }
    io_bytes = b;
    return DPC_OK;
  }
};

// Records CUDA events around one phase when the call asked for phase times.
struct Phase {
  Workspace* w;
  int ph;
  cudaEvent_t a = nullptr;
  Phase(Workspace* w_, int ph_) : w(w_), ph(ph_) {
    if (w->timing) {
      a = w->take_event();
      cudaEventRecord(a, w->stream);
    }
  }
  ~Phase() {
    if (w->timing) {
      cudaEvent_t b = w->take_event();
      cudaEventRecord(b, w->stream);
      w->recs.push_back({ph, a, b});
    }
  }
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

int get_workspace(cudaStream_t st, Workspace** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, st);
  auto it = g_ws.find(key);
  if (it == g_ws.end()) {
    Workspace* w = new Workspace();
    w->device = dev;
    w->stream = st;
    it = g_ws.emplace(key, w).first;
  }
  *out = it->second;
  return DPC_OK;
}

// ---- argument checks -----------------------------------------------------------

struct Inst {
  uint64_t n;
  int d;
  uint64_t pt_off;     // into result arrays
  uint64_t coord_off;  // into pts, in elements
};

int check_batch(const dpc_batch* b, std::vector<Inst>* insts, uint64_t* total) {
  if (!b || b->n_inst < 1 || !b->pt_offset || !b->dim || b->n_dcut < 1 || !b->d_cut) return DPC_ERR_ARG;
  if (b->pt_offset[0] != 0) return DPC_ERR_ARG;
  insts->clear();
  insts->reserve(b->n_inst);
  for (int i = 0; i < b->n_inst; ++i) {
    const int64_t lo = b->pt_offset[i], hi = b->pt_offset[i + 1];
    if (hi < lo) return DPC_ERR_ARG;
    const int d = b->dim[i];
    if (d < 1 || d > kMaxDim) return DPC_ERR_ARG;
    if (hi - lo >= (int64_t)0x7fffffff) return DPC_ERR_OVERFLOW;
    Inst in;
    in.n = (uint64_t)(hi - lo);
    in.d = d;
    in.pt_off = (uint64_t)lo;
    in.coord_off = b->coord_offset ? (uint64_t)b->coord_offset[i] : (uint64_t)lo * (uint64_t)d;
    if (b->coord_offset && b->coord_offset[i] < 0) return DPC_ERR_ARG;
    for (int c = 0; c < b->n_dcut; ++c) {
      const double dc = b->d_cut[(size_t)i * b->n_dcut + c];
      if (!std::isfinite(dc) || dc < 0.0) return DPC_ERR_ARG;
    }
    insts->push_back(in);
  }
  *total = (uint64_t)b->pt_offset[b->n_inst];
  return DPC_OK;
}

int check_flags(uint32_t flags) {
  const uint32_t prec = flags & DPC_PREC_MASK;
  if (prec != DPC_PREC_FP64 && prec != DPC_PREC_FP32_CERT) return DPC_ERR_UNSUPPORTED;
  if (flags & ~(DPC_PREC_MASK | DPC_FLAG_SYNC_CHECK | DPC_FLAG_PHASE_TIMES)) return DPC_ERR_ARG;
  return DPC_OK;
}

inline int dp_of(int d) { return d <= 2 ? 2 : (d <= 4 ? 4 : 8); }
inline int g_of(int d) { return d < 3 ? d : 3; }

int status_to_code(int s) {
  if (s == 0) return DPC_OK;
  if (s & (kStatusBadCoord | kStatusCycle)) return DPC_ERR_DATA;
  if (s & kStatusStack) return DPC_ERR_UNSUPPORTED;
  return DPC_ERR_CUDA;
}

int finish(Workspace* w, uint32_t flags) {
  w->end_call();
  if (cudaGetLastError() != cudaSuccess) return DPC_ERR_CUDA;
  if (flags & DPC_FLAG_SYNC_CHECK) {
    if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    int s = 0;
    if (cudaMemcpy(&s, w->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    return status_to_code(s);
  }
  return DPC_OK;
}

// ---- pipeline pieces --------------------------------------------------------------

// Binning of one instance: geometry for the given cutoffs, sorted points.
void bin_instance(Workspace* w, const void* pts, int dtype, const Inst& in,
                  const std::vector<CutHost>& cuts) {
  cudaStream_t st = w->stream;
  const uint32_t n = (uint32_t)in.n;
  const int d = in.d, g = g_of(d), dp = dp_of(d);
  const size_t esz = 4;
  const void* p = (const char*)pts + in.coord_off * esz;
  Phase ph(w, DPC_PHASE_BIN);
  w->boxes_ready = false;
  launch_geom_init(w->geom, w->status, g, st);
  launch_bbox(p, dtype, n, d, g, w->geom, st);
  launch_setup(w->geom, w->cuts, cuts.data(), (int)cuts.size(), st);
  launch_codes(p, dtype, n, d, w->geom, w->codes_a, w->ids_a, st);
  launch_sort(w->codes_a, w->codes_b, w->ids_a, w->ids_b, n, w->geom, w->hist, st);
  launch_gather(p, dtype, n, d, dp, w->geom, w->codes_a, w->codes_b, w->ids_a, w->ids_b, w->spts,
                w->scode, w->sid, st);
}

std::vector<CutHost> host_cuts(const dpc_batch* b, int inst, int dp, int only = -1) {
  std::vector<CutHost> v;
  for (int c = 0; c < b->n_dcut; ++c) {
    if (only >= 0 && c != only) continue;
    v.push_back(make_cut_host(b->d_cut[(size_t)inst * b->n_dcut + c], dp));
  }
  return v;
}

FarQueue queue_of(Workspace* w) {
  FarQueue q;
  q.pos = w->qpos;
  q.s1 = w->qs1;
  q.s1d = w->qs1d;
  q.pos2 = w->qpos2;
  q.s1_2 = w->qs1_2;
  q.s1d2 = w->qs1d2;
  return q;
}

void dependent_step(Workspace* w, const void* pts_all, int dtype, const Inst& in, CutGeom* cut,
                    int32_t rho_skip, bool fp64, int32_t* lambda, double* delta) {
  const void* pts = (const char*)pts_all + in.coord_off * 4;
  cudaStream_t st = w->stream;
  const uint32_t n = (uint32_t)in.n;
  const int d = in.d, g = g_of(d), dp = dp_of(d);
  {
    Phase ph(w, DPC_PHASE_MAXKEY);
    launch_tree_maxkey(w->skey, w->spts, dp, n, w->nodes, w->leaf_parent, w->visit, w->nbox,
                       !w->boxes_ready, st);
    w->boxes_ready = true;
  }
  {
    Phase ph(w, DPC_PHASE_NEAR);
    launch_dep_near(dp, g, fp64, w->spts, w->scode, w->skey, n, rho_skip, pts, dtype, d, w->geom, cut,
                    w->hkeys, w->hvals, lambda, delta, queue_of(w), w->ctr, st);
  }
  {
    Phase ph(w, DPC_PHASE_FAR);
    launch_dep_far(dp, fp64, w->spts, w->skey, n, w->geom, cut, w->nodes, w->nbox, queue_of(w),
                   lambda, delta, w->ctr, n, st);
  }
}

void cells_step(Workspace* w, uint32_t n, CutGeom* cut) {
  Phase ph(w, DPC_PHASE_CELLS);
  launch_cells(w->scode, n, w->geom, cut, w->hkeys, w->hvals, w->hcap, w->stream);
}

void density_step(Workspace* w, const Inst& in, CutGeom* cut, bool fp64, int32_t* rho) {
  Phase ph(w, DPC_PHASE_DENSITY);
  launch_density(dp_of(in.d), g_of(in.d), fp64, w->spts, w->scode, w->sid, (uint32_t)in.n, w->geom,
                 cut, w->hkeys, w->hvals, rho, w->skey, w->ctr, w->stream);
}

void tree_step(Workspace* w, uint32_t n) {
  Phase ph(w, DPC_PHASE_TREE);
  launch_tree_build(w->scode, n, w->geom, w->nodes, w->leaf_parent, w->stream);
}

void labels_step(Workspace* w, uint32_t n, const dpc_params& P, const int32_t* rho,
                 const int32_t* lambda, const double* delta, int32_t* label) {
  Phase ph(w, DPC_PHASE_LABELS);
  launch_labels(rho, lambda, delta, n, P.rho_noise, P.rho_min, P.delta_min, label, w->flags,
                w->geom, w->stream);
}

uint64_t max_n(const std::vector<Inst>& v) {
  uint64_t m = 0;
  for (auto& i : v) m = i.n > m ? i.n : m;
  return m;
}

void reset_call(Workspace* w, uint32_t flags) {
  w->begin_call(flags);
  cudaMemsetAsync(w->status, 0, sizeof(int), w->stream);
  cudaMemsetAsync(w->ctr, 0, sizeof(Counters), w->stream);
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" {

const char* dpc_version(void) { return "0.1.0"; }

const char* dpc_strerror(int status) {
  switch (status) {
    case DPC_OK: return "ok";
    case DPC_ERR_ARG: return "invalid argument";
    case DPC_ERR_CUDA: return "CUDA error or no CUDA device";
    case DPC_ERR_OOM: return "device memory allocation failed";
    case DPC_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case DPC_ERR_OVERFLOW: return "an instance has 2^31 or more points";
    case DPC_ERR_UNSUPPORTED: return "not supported by this build";
    case DPC_ERR_DATA: return "coordinates out of range or NaN, or dependent pointers not a forest";
    default: return "unknown status";
  }
}

int dpc_density(const void* pts, int dtype, const dpc_batch* b, int32_t* rho, uint32_t flags,
                void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_batch(b, &insts, &N);
  if (rc) return rc;
  if ((rc = check_flags(flags))) return rc;
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (N > 0 && (!pts || !rho)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((rc = w->reserve(max_n(insts), b->n_dcut))) return rc;
  reset_call(w, flags);
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  for (int i = 0; i < b->n_inst; ++i) {
    const Inst& in = insts[i];
    if (in.n == 0) continue;
    const int dp = dp_of(in.d);
    std::vector<CutHost> cuts = host_cuts(b, i, dp);
    bin_instance(w, pts, dtype, in, cuts);
    for (int c = 0; c < b->n_dcut; ++c) {
      cells_step(w, (uint32_t)in.n, w->cuts + c);
      density_step(w, in, w->cuts + c, fp64, rho + (size_t)c * N + in.pt_off);
    }
    w->last_ncut_used = b->n_dcut;
  }
  return finish(w, flags);
}

int dpc_dependent(const void* pts, int dtype, const dpc_batch* b, int32_t dcut_index,
                  const int32_t* rho, int32_t rho_skip, int32_t* lambda, double* delta,
                  uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_batch(b, &insts, &N);
  if (rc) return rc;
  if ((rc = check_flags(flags))) return rc;
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (dcut_index < 0 || dcut_index >= b->n_dcut) return DPC_ERR_ARG;
  if (N > 0 && (!pts || !rho || !lambda || !delta)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((rc = w->reserve(max_n(insts), 1))) return rc;
  reset_call(w, flags);
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  for (int i = 0; i < b->n_inst; ++i) {
    const Inst& in = insts[i];
    if (in.n == 0) continue;
    const int dp = dp_of(in.d);
    std::vector<CutHost> cuts = host_cuts(b, i, dp, dcut_index);
    bin_instance(w, pts, dtype, in, cuts);
    tree_step(w, (uint32_t)in.n);
    cells_step(w, (uint32_t)in.n, w->cuts);
    launch_keys_from_rho(rho + in.pt_off, w->sid, (uint32_t)in.n, w->skey, w->stream);
    dependent_step(w, pts, dtype, in, w->cuts, rho_skip, fp64, lambda + in.pt_off, delta + in.pt_off);
    w->last_ncut_used = 1;
  }
  return finish(w, flags);
}

int dpc_cluster(const dpc_batch* b, int32_t dcut_index, const dpc_params* params,
                const int32_t* rho, const int32_t* lambda, const double* delta, int32_t* label,
                uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_batch(b, &insts, &N);
  if (rc) return rc;
  if (flags & ~(DPC_PREC_MASK | DPC_FLAG_SYNC_CHECK | DPC_FLAG_PHASE_TIMES)) return DPC_ERR_ARG;
  if (dcut_index < 0 || dcut_index >= b->n_dcut || !params) return DPC_ERR_ARG;
  if (N > 0 && (!rho || !lambda || !delta || !label)) return DPC_ERR_ARG;
  for (int i = 0; i < b->n_inst; ++i)
    if (std::isnan(params[(size_t)i * b->n_dcut + dcut_index].delta_min)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((rc = w->reserve(max_n(insts), 1))) return rc;
  reset_call(w, flags);
  for (int i = 0; i < b->n_inst; ++i) {
    const Inst& in = insts[i];
    if (in.n == 0) continue;
    const dpc_params& P = params[(size_t)i * b->n_dcut + dcut_index];
    launch_geom_init(w->geom, w->status, g_of(in.d), w->stream);
    labels_step(w, (uint32_t)in.n, P, rho + in.pt_off, lambda + in.pt_off, delta + in.pt_off,
                label + in.pt_off);
  }
  return finish(w, flags);
}

static int run_device(Workspace* w, const void* pts, int dtype, const dpc_batch* b,
                      const std::vector<Inst>& insts, uint64_t N, const dpc_params* params,
                      int32_t* rho, int32_t* lambda, double* delta, int32_t* label,
                      uint32_t flags) {
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  reset_call(w, flags);
  for (int i = 0; i < b->n_inst; ++i) {
    const Inst& in = insts[i];
    if (in.n == 0) continue;
    const uint32_t n = (uint32_t)in.n;
    const int dp = dp_of(in.d);
    std::vector<CutHost> cuts = host_cuts(b, i, dp);
    bin_instance(w, pts, dtype, in, cuts);
    tree_step(w, n);
    for (int c = 0; c < b->n_dcut; ++c) {
      const size_t o = (size_t)c * N + in.pt_off;
      CutGeom* cut = w->cuts + c;
      cells_step(w, n, cut);
      density_step(w, in, cut, fp64, rho + o);
      dependent_step(w, pts, dtype, in, cut, 0, fp64, lambda + o, delta + o);
      labels_step(w, n, params[(size_t)i * b->n_dcut + c], rho + o, lambda + o, delta + o, label + o);
    }
    w->last_ncut_used = b->n_dcut;
  }
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}

static int check_run(const void* pts, int dtype, const dpc_batch* b, const dpc_params* params,
                     const void* rho, const void* lambda, const void* delta, const void* label,
                     uint32_t flags, std::vector<Inst>* insts, uint64_t* N) {
  int rc = check_batch(b, insts, N);
  if (rc) return rc;
  if ((rc = check_flags(flags))) return rc;
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (!params) return DPC_ERR_ARG;
  for (int i = 0; i < b->n_inst * b->n_dcut; ++i)
    if (std::isnan(params[i].delta_min)) return DPC_ERR_ARG;
  if (*N > 0 && (!pts || !rho || !lambda || !delta || !label)) return DPC_ERR_ARG;
  return DPC_OK;
}

int dpc_run(const void* pts, int dtype, const dpc_batch* b, const dpc_params* params, int32_t* rho,
            int32_t* lambda, double* delta, int32_t* label, uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_run(pts, dtype, b, params, rho, lambda, delta, label, flags, &insts, &N);
  if (rc) return rc;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((rc = w->reserve(max_n(insts), b->n_dcut))) return rc;
  if ((rc = run_device(w, pts, dtype, b, insts, N, params, rho, lambda, delta, label, flags))) return rc;
  return finish(w, flags);
}

int dpc_run_host(const void* pts_host, int dtype, const dpc_batch* b, const dpc_params* params,
                 int32_t* rho_host, int32_t* lambda_host, double* delta_host, int32_t* label_host,
                 uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_run(pts_host, dtype, b, params, rho_host, lambda_host, delta_host, label_host,
                     flags, &insts, &N);
  if (rc) return rc;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((rc = w->reserve(max_n(insts), b->n_dcut))) return rc;
  uint64_t elems = 0;
  for (auto& in : insts) {
    uint64_t e = in.coord_off + in.n * (uint64_t)in.d;
    elems = e > elems ? e : elems;
  }
  const size_t R = (size_t)b->n_dcut * N;
  const size_t o_pts = 0;
  const size_t o_rho = align_up(4 * elems);
  const size_t o_lam = o_rho + align_up(4 * R);
  const size_t o_del = o_lam + align_up(4 * R);
  const size_t o_lab = o_del + align_up(8 * R);
  const size_t total = o_lab + align_up(4 * R);
  if ((rc = w->reserve_io(total ? total : kAlign))) return rc;
  char* io = (char*)w->io;
  cudaStream_t st = w->stream;
  if (elems) cudaMemcpyAsync(io + o_pts, pts_host, 4 * elems, cudaMemcpyHostToDevice, st);
  rc = run_device(w, io + o_pts, dtype, b, insts, N, params, (int32_t*)(io + o_rho),
                  (int32_t*)(io + o_lam), (double*)(io + o_del), (int32_t*)(io + o_lab), flags);
  if (rc) return rc;
  if (R) {
    cudaMemcpyAsync(rho_host, io + o_rho, 4 * R, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(lambda_host, io + o_lam, 4 * R, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(delta_host, io + o_del, 8 * R, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(label_host, io + o_lab, 4 * R, cudaMemcpyDeviceToHost, st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return finish(w, flags | DPC_FLAG_SYNC_CHECK);
}

int dpc_get_stats(void* stream, dpc_stats* out) {
  if (!out) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  int rc = get_workspace((cudaStream_t)stream, &w);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  std::memset(out, 0, sizeof(*out));
  if (!w->base) return DPC_OK;
  if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  Counters c;
  GridGeom g;
  cudaMemcpy(&c, w->ctr, sizeof(c), cudaMemcpyDeviceToHost);
  cudaMemcpy(&g, w->geom, sizeof(g), cudaMemcpyDeviceToHost);
  out->band_pairs = (int64_t)c.band_pairs;
  out->far_queries = (int64_t)c.far_queries;
  out->exact_rescans = (int64_t)c.exact_rescans;
  out->bits_per_axis = g.B;
  out->kernel_launches = w->launches_last;
  out->far_nodes = (int64_t)c.far_nodes;
  out->far_nodes_max = (int64_t)c.far_nodes_max;
  if (w->last_ncut_used > 0) {
    CutGeom cg;
    cudaMemcpy(&cg, w->cuts + (w->last_ncut_used - 1), sizeof(cg), cudaMemcpyDeviceToHost);
    out->occupied_cells = cg.m;
    out->grid_level = cg.k;
  }
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}

int dpc_get_phase_times(void* stream, dpc_phase_times* out) {
  if (!out) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  int rc = get_workspace((cudaStream_t)stream, &w);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  std::memset(out, 0, sizeof(*out));
  if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  for (const auto& r : w->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    out->ms[r.phase] += ms;
    out->launches[r.phase] += 1;
  }
  return DPC_OK;
}

int dpc_last_status(void* stream) {
  Workspace* w = nullptr;
  int rc = get_workspace((cudaStream_t)stream, &w);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!w->base) return DPC_OK;
  if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  int s = 0;
  if (cudaMemcpy(&s, w->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
  }
  return status_to_code(s);
}

void dpc_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_ws) {
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.second->device);
    kv.second->release();
    delete kv.second;
    if (cur >= 0) cudaSetDevice(cur);
  }
  g_ws.clear();
}

}  // extern "C"
