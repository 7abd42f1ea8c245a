// api.cu -- the C ABI (include/dpc.h): argument checks, the per-(device,
// stream) workspace, and the order in which the kernels run.
//
// The instances of a call are grouped into classes of equal padded dimension
// dp and gridded dimension g (at most five: (2,1), (2,2), (4,3), (4,4), (8,4)).  Each
// class runs as one unit, every kernel launched once for all its instances
// (dpc_device.cuh describes the layout):
//   binning   bbox -> grid setup -> sort keys -> radix sort -> gather
//   tree      radix tree over the sorted keys (dependent points only)
//   per cutoff
//     cells     occupied level-k cells -> hash
//     density   rho (Definition 1) + order keys
//     dependent maxkeys of the tree -> near phase -> far phase (Definitions 2-3)
//     labels    pointer jumping (Definitions 4-5)
// All on the caller's stream, with no host synchronization; a multi-instance
// class first copies its instance table and cutoffs to the device (one
// asynchronous copy per call from a page-locked staging buffer).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/dpc.h"
#include "internal.h"

namespace dpc {

long long g_kernel_launches = 0;

uint32_t wait_limit(uint32_t dflt) {
  const char* e = std::getenv("DPC_TEST_WAIT_LIMIT");
  if (!e || !*e) return dflt;
  char* end = nullptr;
  const unsigned long long v = std::strtoull(e, &end, 10);
  if (end == e) return dflt;
  return v < dflt ? (uint32_t)v : dflt;
}

bool dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  const char* e = std::getenv("DPC_WORKSPACE_LIMIT_BYTES");
  if (e && *e) {
    char* end = nullptr;
    const unsigned long long cap = std::strtoull(e, &end, 10);
    if (end != e && bytes > cap) return false;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

unsigned sm_count() {
  constexpr int kDevs = 64;
  static int cached[kDevs] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
    cudaGetLastError();
    return 1u;  // the launch that follows reports the error
  }
  if (cached[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      return 1u;
    }
    cached[dev] = v;
  }
  return (unsigned)cached[dev];
}

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

inline uint32_t next_pow2(uint64_t x) {
  uint64_t t = 16;
  while (t < x) t <<= 1;
  return (uint32_t)t;
}

inline int dp_of(int d) { return d <= 2 ? 2 : (d <= 4 ? 4 : 8); }
inline int g_of(int d) { return grid_dims(d); }

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
  // output indices are 32-bit inside the library
  if (b->pt_offset[b->n_inst] >= (int64_t)0x7fffffff) return DPC_ERR_OVERFLOW;
  *total = (uint64_t)b->pt_offset[b->n_inst];
  return DPC_OK;
}

constexpr uint32_t kKnownFlags = DPC_PREC_MASK | DPC_FLAG_SYNC_CHECK | DPC_FLAG_PHASE_TIMES |
                                 DPC_FLAG_AUTOTUNE | DPC_FLAG_RADIUS_MASK | DPC_FLAG_GRAPH |
                                 DPC_FLAG_LAYOUT_MASK | DPC_FLAG_SKIP_NOISE |
                                 DPC_FLAG_NEAR_SHIFT_MASK;

int check_flags(uint32_t flags) {
  const uint32_t prec = flags & DPC_PREC_MASK;
  if (prec != DPC_PREC_FP64 && prec != DPC_PREC_FP32_CERT) return DPC_ERR_UNSUPPORTED;
  if (flags & ~kKnownFlags) return DPC_ERR_ARG;
  if (((flags & DPC_FLAG_RADIUS_MASK) >> 12) > 5) return DPC_ERR_ARG;
  if (((flags & DPC_FLAG_LAYOUT_MASK) >> 16) > 6) return DPC_ERR_ARG;
  if (((flags & DPC_FLAG_NEAR_SHIFT_MASK) >> 20) > 3) return DPC_ERR_ARG;
  return DPC_OK;
}

int status_to_code(int s) {
  if (s == 0) return DPC_OK;
  if (s & kStatusBadCoord) return DPC_ERR_DATA;
  // a wait that gave up leaves later results unreliable: report it first
  if (s & kStatusTimeout) return DPC_ERR_TIMEOUT;
  if (s & (kStatusCycle | kStatusQuery)) return DPC_ERR_DATA;
  if (s & kStatusStack) return DPC_ERR_UNSUPPORTED;
  return DPC_ERR_CUDA;
}

// ---- classes -------------------------------------------------------------------

// One class of a call: the non-empty instances sharing (dp, g), in batch order.
struct ClassPlan {
  int dp = 0, g = 0;
  std::vector<int> members;  // batch indices
  uint32_t N = 0, nchunk = 0, nmax = 0;
  int ib = 0, bcap = kMaxBits;
  // offsets of this class's tables in the upload block (multi-instance only)
  size_t off_inst = 0, off_cut = 0, off_par = 0;
  // tables on the device (several instances, or more cutoffs than fit in
  // kernel arguments); a single instance otherwise runs without them
  bool upload = false;
  bool uploaded() const { return upload; }
};

// Groups the instances into classes; `all_one` puts every instance in one
// class (labels only, where the dimension does not matter).
std::vector<ClassPlan> plan_classes(const std::vector<Inst>& insts, bool all_one) {
  std::vector<ClassPlan> out;
  const int keys[5][2] = {{2, 1}, {2, 2}, {4, 3}, {4, 4}, {8, 4}};
  for (int k = 0; k < (all_one ? 1 : 5); ++k) {
    ClassPlan c;
    c.dp = keys[k][0];
    c.g = keys[k][1];
    for (size_t i = 0; i < insts.size(); ++i) {
      const Inst& in = insts[i];
      if (in.n == 0) continue;
      if (!all_one && (dp_of(in.d) != c.dp || g_of(in.d) != c.g)) continue;
      c.members.push_back((int)i);
      c.N += (uint32_t)in.n;
      c.nchunk += (uint32_t)((in.n + 31) / 32);
      c.nmax = std::max(c.nmax, (uint32_t)in.n);
    }
    if (c.members.empty()) continue;
    int ib = 0;
    while ((size_t(1) << ib) < c.members.size()) ++ib;
    c.ib = ib;
    c.bcap = std::min(kMaxBits, (63 - ib) / c.g);
    out.push_back(std::move(c));
  }
  return out;
}

// Grid level and kernel layouts chosen for one (class, cutoff); r = 0: the
// default rule.
struct Choice {
  int r = 0;
  int dlay = 0;  // density layout (kLayout*)
  int nlay = 0;  // near-phase layout
  int ns = 0;    // near-phase grid levels below the density's
  int sc = 0;    // segment layouts: cells a segment's union may hold (0: one cell)
};

struct Workspace {
  int device = -1;
  cudaStream_t stream = nullptr;
  uint64_t cap_n = 0;     // points per class the buffers hold
  uint32_t cap_inst = 0;  // instances per class
  int cap_ncut = 0;
  void* base = nullptr;   // one allocation, carved below
  size_t bytes = 0;

  GridGeom* geom = nullptr;   // [cap_inst]
  CutGeom* cuts = nullptr;    // [cap_ncut][cap_inst]
  ClassGeom* cls = nullptr;
  HashInfo* hinfo = nullptr;
  Counters* ctr = nullptr;
  Counters* ctr_save = nullptr;  // the counters during autotuning trials
  int* status = nullptr;
  int32_t* flags = nullptr;
  uint32_t* roots = nullptr;  // [cap_inst]
  uint32_t* chunk_inst = nullptr;
  uint32_t* chunk_pos = nullptr;
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
  float* nbox = nullptr;    // per-node child records of the radix tree (dpc_device.cuh)
  bool boxes_ready = false; // nbox matches the current binning
  uint32_t* leaf_parent = nullptr;
  uint32_t* visit = nullptr;
  uint2* pieces = nullptr;        // 128-point pieces of the cells (tensor-core density)
  uint32_t* qpos = nullptr;
  float* qs1 = nullptr;
  double* qs1d = nullptr;
  uint32_t* qpos2 = nullptr;
  float* qs1_2 = nullptr;
  double* qs1d2 = nullptr;

  // instance tables and cutoffs of multi-instance classes: filled in the
  // page-locked host buffer, copied to the device buffer once per call
  void* up_dev = nullptr;
  void* up_host = nullptr;
  size_t up_bytes = 0;
  cudaEvent_t up_done = nullptr;  // the last copy out of up_host has finished

  // host-buffer entry point staging; its copies to the host run on a stream
  // of their own, each behind the event of the phase that finished its output
  void* io = nullptr;
  size_t io_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> out_ev;

  // priority range search: per-query arrays (scr) and the match keys (scr2)
  void* scr = nullptr;
  size_t scr_bytes = 0;
  void* scr2 = nullptr;
  size_t scr2_bytes = 0;

  // the captured graph of DPC_FLAG_GRAPH calls and the key it was captured for
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  long long glaunches = 0;
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    gkey.clear();
  }

  // autotuned radius and layouts per (class shape, cutoff), see choose()
  std::map<std::string, Choice> tuned;
  cudaEvent_t tune_ev[24] = {};

  // for dpc_get_stats: the last class and cutoff that ran
  Choice last_choice;
  const CutGeom* last_cut = nullptr;
  const GridGeom* last_geom = nullptr;
  bool have_last = false;
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

  void begin_call(uint32_t fl) {
    timing = (fl & DPC_FLAG_PHASE_TIMES) != 0;
    recs.clear();
    ev_used = 0;
    g_kernel_launches = 0;
  }
  void end_call() { launches_last = g_kernel_launches; }

  void release() {
    drop_graph();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    ev_used = 0;
    recs.clear();
    if (base) cudaFree(base);
    if (io) cudaFree(io);
    if (scr) cudaFree(scr);
    if (scr2) cudaFree(scr2);
    scr = scr2 = nullptr;
    scr_bytes = scr2_bytes = 0;
    if (up_dev) cudaFree(up_dev);
    if (up_host) cudaFreeHost(up_host);
    if (up_done) cudaEventDestroy(up_done);
    for (cudaEvent_t e : out_ev) cudaEventDestroy(e);
    out_ev.clear();
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    for (auto& e : tune_ev) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    base = io = up_dev = up_host = nullptr;
    up_done = nullptr;
    tuned.clear();
    bytes = io_bytes = up_bytes = 0;
    cap_n = 0;
    cap_inst = 0;
    cap_ncut = 0;
    have_last = false;
  }

  int reserve(uint64_t n, uint32_t ninst, int ncut) {
    if (n <= cap_n && ninst <= cap_inst && ncut <= cap_ncut && base) return DPC_OK;
    uint64_t want_n = std::max<uint64_t>(std::max<uint64_t>(n, cap_n), 1024);
    uint32_t want_i = std::max<uint32_t>(std::max<uint32_t>(ninst, cap_inst), 1);
    int want_c = std::max(std::max(ncut, cap_ncut), 8);
    if (base) {
      cudaStreamSynchronize(stream);
      drop_graph();  // it holds pointers into the old buffers
      cudaFree(base);
      base = nullptr;
    }
    const uint64_t N = want_n;
    const uint32_t hc = next_pow2(2 * N);
    const uint64_t nchunk = N / 32 + want_i + 1;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align_up(b); return o; };
    const size_t o_geom = take(sizeof(GridGeom) * want_i);
    const size_t o_cuts = take(sizeof(CutGeom) * want_i * (size_t)want_c);
    const size_t o_cls = take(sizeof(ClassGeom));
    const size_t o_hi = take(sizeof(HashInfo));
    const size_t o_ctr = take(sizeof(Counters));
    const size_t o_ctr2 = take(sizeof(Counters));
    const size_t o_status = take(sizeof(int));
    const size_t o_flags = take(sizeof(int32_t) * 80);
    const size_t o_roots = take(sizeof(uint32_t) * want_i);
    const size_t o_ci = take(4 * nchunk), o_cp = take(4 * nchunk);
    const size_t o_ca = take(8 * N), o_cb = take(8 * N);
    const size_t o_ia = take(4 * N), o_ib = take(4 * N);
    const size_t o_hist = take(4 * sort_hist_words((uint32_t)N));
    const size_t o_spts = take(4 * 8 * N);
    const size_t o_scode = take(8 * N);
    const size_t o_sid = take(4 * N);
    const size_t o_skey = take(8 * N);
    const size_t o_hk = take(8 * (size_t)hc), o_hv = take(8 * (size_t)hc);
    const size_t o_nodes = take(sizeof(Node) * N);
    const size_t o_nbox = take(4 * (size_t)kRecWordsMax * N);
    const size_t o_lp = take(4 * N), o_visit = take(4 * N);
    const size_t o_pieces = take(8 * N);
    const size_t o_qpos = take(4 * N), o_qs1 = take(4 * N), o_qs1d = take(8 * N);
    const size_t o_qpos2 = take(4 * N), o_qs1_2 = take(4 * N), o_qs1d2 = take(8 * N);
    void* p = nullptr;
    if (!dev_alloc(&p, off)) {
      cap_n = 0;
      cap_inst = 0;
      return DPC_ERR_OOM;
    }
    base = p;
    bytes = off;
    char* b = (char*)p;
    geom = (GridGeom*)(b + o_geom);
    cuts = (CutGeom*)(b + o_cuts);
    cls = (ClassGeom*)(b + o_cls);
    hinfo = (HashInfo*)(b + o_hi);
    ctr = (Counters*)(b + o_ctr);
    ctr_save = (Counters*)(b + o_ctr2);
    status = (int*)(b + o_status);
    flags = (int32_t*)(b + o_flags);
    roots = (uint32_t*)(b + o_roots);
    chunk_inst = (uint32_t*)(b + o_ci);
    chunk_pos = (uint32_t*)(b + o_cp);
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
    pieces = (uint2*)(b + o_pieces);
    qpos = (uint32_t*)(b + o_qpos);
    qs1 = (float*)(b + o_qs1);
    qs1d = (double*)(b + o_qs1d);
    qpos2 = (uint32_t*)(b + o_qpos2);
    qs1_2 = (float*)(b + o_qs1_2);
    qs1d2 = (double*)(b + o_qs1d2);
    cap_n = N;
    cap_inst = want_i;
    cap_ncut = want_c;
    have_last = false;
    cudaMemsetAsync(status, 0, sizeof(int), stream);
    cudaMemsetAsync(ctr, 0, sizeof(Counters), stream);
    return DPC_OK;
  }

  // Makes the upload buffers at least `b` bytes and waits until the previous
  // copy out of the host buffer has finished, so it can be rewritten.
  int reserve_upload(size_t b) {
    if (!up_done) {
      if (cudaEventCreateWithFlags(&up_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return DPC_ERR_CUDA;
      }
    } else if (cudaEventSynchronize(up_done) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    if (b <= up_bytes && up_dev) return DPC_OK;
    if (up_dev) {
      cudaStreamSynchronize(stream);
      drop_graph();
      cudaFree(up_dev);
      cudaFreeHost(up_host);
      up_dev = up_host = nullptr;
      up_bytes = 0;
    }
    if (!dev_alloc(&up_dev, b)) return DPC_ERR_OOM;
    if (cudaMallocHost(&up_host, b) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(up_dev);
      up_dev = up_host = nullptr;
      return DPC_ERR_OOM;
    }
    up_bytes = b;
    return DPC_OK;
  }

  // grow-only device scratch (contents not kept across growth)
  int reserve_buf(void** p, size_t* have, size_t b) {
    if (b <= *have && *p) return DPC_OK;
    if (*p) {
      cudaStreamSynchronize(stream);
      cudaFree(*p);
      *p = nullptr;
    }
    if (!dev_alloc(p, b)) {
      *have = 0;
      return DPC_ERR_OOM;
    }
    *have = b;
    return DPC_OK;
  }

  int reserve_io(size_t b) {
    if (b <= io_bytes && io) return DPC_OK;
    if (io) {
      cudaStreamSynchronize(stream);
      cudaFree(io);
      io = nullptr;
    }
    if (!dev_alloc(&io, b)) {
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

// ---- one call: plan, upload, classes ----------------------------------------------

// What a call runs.  cut_first/ncut select the cutoffs (all, or one);
// params (may be null) are the labelling thresholds.
struct CallPlan {
  std::vector<ClassPlan> classes;
  int ncut_all = 1;   // n_dcut of the batch
  int cut_first = 0;  // first cutoff this call uses
  int ncut = 1;       // cutoffs this call uses
  uint32_t max_inst = 0;
  uint64_t max_n = 0;
  const dpc_params* params = nullptr;  // thresholds of the call (dpc_run, dpc_cluster)
  bool skip_noise = false;             // DPC_FLAG_SKIP_NOISE
};

CallPlan make_plan(const dpc_batch* b, const std::vector<Inst>& insts, int cut_first, int ncut,
                   bool all_one) {
  CallPlan P;
  P.classes = plan_classes(insts, all_one);
  P.ncut_all = b->n_dcut;
  P.cut_first = cut_first;
  P.ncut = ncut;
  for (auto& c : P.classes) {
    c.upload = c.members.size() > 1 || ncut > kCutChunk;
    P.max_inst = std::max<uint32_t>(P.max_inst, (uint32_t)c.members.size());
    P.max_n = std::max<uint64_t>(P.max_n, c.N);
  }
  return P;
}

// The cutoff constants of (instance bi, cutoff cut); with DPC_FLAG_SKIP_NOISE
// the dependent search skips that pair's noise points.
CutHost cut_host(const CallPlan& P, const dpc_batch* b, int bi, int cut, int dp) {
  CutHost h = make_cut_host(b->d_cut[(size_t)bi * P.ncut_all + cut], dp);
  if (P.skip_noise && P.params) h.skip = P.params[(size_t)bi * P.ncut_all + cut].rho_noise;
  return h;
}

// Fills and copies the tables of every multi-instance class (instance
// descriptors, cutoff constants [inst][cut], label thresholds [cut][inst]).
int upload_tables(Workspace* w, CallPlan& P, const dpc_batch* b, const std::vector<Inst>& insts,
                  const dpc_params* params) {
  size_t total = 0;
  for (auto& c : P.classes) {
    if (!c.uploaded()) continue;
    const size_t m = c.members.size();
    c.off_inst = total;
    total += align_up(sizeof(InstDev) * m);
    c.off_cut = total;
    total += align_up(sizeof(CutHost) * m * P.ncut);
    c.off_par = total;
    total += align_up(sizeof(LabelParams) * m * P.ncut);
  }
  if (total == 0) return DPC_OK;
  int rc = w->reserve_upload(total);
  if (rc) return rc;
  char* h = (char*)w->up_host;
  for (auto& c : P.classes) {
    if (!c.uploaded()) continue;
    const size_t m = c.members.size();
    InstDev* id = (InstDev*)(h + c.off_inst);
    CutHost* ch = (CutHost*)(h + c.off_cut);
    LabelParams* lp = (LabelParams*)(h + c.off_par);
    uint32_t start = 0, chunk = 0;
    for (size_t j = 0; j < m; ++j) {
      const int bi = c.members[j];
      const Inst& in = insts[bi];
      id[j].start = start;
      id[j].n = (uint32_t)in.n;
      id[j].out = in.pt_off;
      id[j].coord = in.coord_off;
      id[j].d = in.d;
      id[j].chunk0 = chunk;
      id[j].row = (uint32_t)bi;
      id[j].pad = 0;
      start += (uint32_t)in.n;
      chunk += (uint32_t)((in.n + 31) / 32);
      for (int k = 0; k < P.ncut; ++k) {
        const int cut = P.cut_first + k;
        ch[j * P.ncut + k] = cut_host(P, b, bi, cut, c.dp);
        LabelParams L{0, 0, 0.0};
        if (params) {
          const dpc_params& q = params[(size_t)bi * P.ncut_all + cut];
          L.rho_noise = q.rho_noise;
          L.rho_min = q.rho_min;
          L.delta_min = q.delta_min;
        }
        lp[(size_t)k * m + j] = L;
      }
    }
  }
  cudaMemcpyAsync(w->up_dev, w->up_host, total, cudaMemcpyHostToDevice, w->stream);
  cudaEventRecord(w->up_done, w->stream);
  return DPC_OK;
}

// The device view of one class.
ClassView view_of(Workspace* w, const ClassPlan& c, const std::vector<Inst>& insts) {
  ClassView v;
  std::memset(&v, 0, sizeof(v));
  v.N = c.N;
  v.ninst = (uint32_t)c.members.size();
  v.nchunk = c.nchunk;
  v.geom = w->geom;
  v.cls = w->cls;
  if (c.uploaded()) {
    v.inst = (const InstDev*)((char*)w->up_dev + c.off_inst);
    v.chunk_inst = w->chunk_inst;
    v.chunk_pos = w->chunk_pos;
  } else {
    const Inst& in = insts[c.members[0]];
    v.one.start = 0;
    v.one.n = (uint32_t)in.n;
    v.one.out = in.pt_off;
    v.one.coord = in.coord_off;
    v.one.d = in.d;
    v.one.chunk0 = 0;
    v.one.row = (uint32_t)c.members[0];
  }
  return v;
}

const CutHost* cut_table(Workspace* w, const ClassPlan& c) {
  return c.uploaded() ? (const CutHost*)((char*)w->up_dev + c.off_cut) : nullptr;
}

// Binning of one class: geometry for the call's cutoffs, sorted points.
void bin_class(Workspace* w, const void* pts, int dtype, const CallPlan& P, const ClassPlan& c,
               const ClassView& cv, const dpc_batch* b, const std::vector<Inst>& insts) {
  cudaStream_t st = w->stream;
  Phase ph(w, DPC_PHASE_BIN);
  w->boxes_ready = false;
  launch_class_init(cv, c.g, c.ib, c.bcap, w->status, st);
  launch_chunks(cv, w->chunk_inst, w->chunk_pos, st);
  launch_bbox(pts, dtype, cv, c.g, st);
  std::vector<CutHost> hc;
  if (!c.uploaded()) {
    const int bi = c.members[0];
    for (int k = 0; k < P.ncut && k < kCutChunk; ++k)
      hc.push_back(cut_host(P, b, bi, P.cut_first + k, c.dp));
  }
  launch_setup(cv, w->cuts, P.ncut, cut_table(w, c), hc.data(), st);
  launch_codes(pts, dtype, cv, c.g, w->codes_a, w->ids_a, st);
  launch_sort(w->codes_a, w->codes_b, w->ids_a, w->ids_b, cv.N, w->cls, w->hist, st);
  launch_gather(pts, dtype, cv, c.dp, w->codes_a, w->codes_b, w->ids_a, w->ids_b, w->spts,
                w->scode, w->sid, st);
  (void)insts;
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

void tree_step(Workspace* w, const ClassView& cv) {
  Phase ph(w, DPC_PHASE_TREE);
  launch_tree_build(w->scode, cv, w->nodes, w->leaf_parent, w->roots, w->stream);
}

void cells_step(Workspace* w, const ClassPlan& c, const ClassView& cv, const CutGeom* cuts) {
  Phase ph(w, DPC_PHASE_CELLS);
  launch_cells(w->scode, cv, c.g, cuts, w->hinfo, w->hkeys, w->hvals, w->hcap, w->stream);
  w->last_cut = cuts;
  w->last_geom = w->geom;
  w->have_last = true;
}

void density_step(Workspace* w, const ClassPlan& c, const ClassView& cv, const CutGeom* cuts,
                  bool fp64, int layout, int seg_cells, int32_t* rho) {
  Phase ph(w, DPC_PHASE_DENSITY);
  // the tensor layout exists for 5-8 dimensions with the float32 filter;
  // other cases run in segments, and the statistics report what ran
  if (layout == kLayoutTensor && !(c.dp == 8 && !fp64)) layout = kLayoutSegment;
  w->last_choice.dlay = layout;
  launch_density(c.dp, c.g, fp64, layout, w->spts, w->scode, w->sid, cv, cuts, w->hinfo, w->hkeys,
                 w->hvals, w->pieces, rho, w->skey, w->ctr, w->stream, seg_cells);
}

void dependent_step(Workspace* w, const ClassPlan& c, const ClassView& cv, CutGeom* cuts,
                    const void* pts, int dtype, int32_t rho_skip, bool fp64, int layout, int nshift,
                    int seg_cells, int32_t* lambda, double* delta) {
  cudaStream_t st = w->stream;
  {
    Phase ph(w, DPC_PHASE_MAXKEY);
    launch_tree_maxkey(w->skey, w->spts, c.dp, cv.N, w->nodes, w->leaf_parent, w->visit, w->nbox,
                       !w->boxes_ready, st);
    w->boxes_ready = true;
  }
  if (nshift > 0 && layout != kLayoutTree) {  // the near phase on finer cells
    launch_near_level(cv, cuts, nshift, st);
    cells_step(w, c, cv, cuts);
  }
  {
    Phase ph(w, DPC_PHASE_NEAR);
    if (layout == kLayoutTensor && c.dp == 8 && !fp64) {
      launch_dep_near_tc(c.g, w->spts, w->sid, w->skey, cv, rho_skip, pts, dtype, cuts, w->hinfo,
                         w->hkeys, w->hvals, w->pieces, lambda, delta, queue_of(w), w->ctr, st);
    } else {
      // the tensor layout exists for 5-8 dimensions with the float32 filter
      if (layout == kLayoutTensor) layout = kLayoutUnion;
      launch_dep_near(c.dp, c.g, fp64, layout, w->spts, w->scode, w->skey, cv, rho_skip, pts, dtype,
                      cuts, w->hinfo, w->hkeys, w->hvals, lambda, delta, queue_of(w), w->ctr, st,
                      seg_cells);
    }
    w->last_choice.nlay = layout;
  }
  {
    Phase ph(w, DPC_PHASE_FAR);
    launch_dep_far(c.dp, fp64, w->spts, w->scode, w->skey, cv, cuts, w->nodes, w->nbox, w->roots,
                   queue_of(w), lambda, delta, w->ctr, st);
  }
}

void labels_step(Workspace* w, const ClassPlan& c, const ClassView& cv, int k_in_call,
                 const LabelParams& one, const int32_t* rho, const int32_t* lambda,
                 const double* delta, int32_t* label) {
  Phase ph(w, DPC_PHASE_LABELS);
  const LabelParams* par =
      c.uploaded()
          ? (const LabelParams*)((char*)w->up_dev + c.off_par) + (size_t)k_in_call * c.members.size()
          : nullptr;
  launch_labels(rho, lambda, delta, cv, c.nmax, par, one, label, w->flags, w->stream);
}

LabelParams one_params(const dpc_params* params, const ClassPlan& c, int ncut_all, int cut) {
  LabelParams L{0, 0, 0.0};
  if (params && !c.uploaded()) {
    const dpc_params& q = params[(size_t)c.members[0] * ncut_all + cut];
    L.rho_noise = q.rho_noise;
    L.rho_min = q.rho_min;
    L.delta_min = q.delta_min;
  }
  return L;
}

// ---- autotuning of the cell level -------------------------------------------------
//
// The block radius R (and with it the grid level: finer cells for larger R)
// decides how many candidates a query scans and how many cells a warp looks
// up.  The default rule keeps R = 1 unless a larger R shrinks the block side
// by 20%; with DPC_FLAG_AUTOTUNE the first call for a class shape times the
// density step once per radius (R = 1, 2, 3 in 1-2 gridded dims, R = 1, 2 in
// 3; 4 gridded dims allow only R = 1) and keeps the fastest for later calls of
// the same shape.

std::string tune_key(const ClassPlan& c, const dpc_batch* b, int cut) {
  char buf[160];
  const double dc = b->d_cut[(size_t)c.members[0] * b->n_dcut + cut];
  unsigned long long bits;
  std::memcpy(&bits, &dc, sizeof(bits));
  std::snprintf(buf, sizeof(buf), "%d/%d/%zu/%u/%d/%llx", c.dp, c.g, c.members.size(), c.N, cut, bits);
  return buf;
}

// What a tuning trial of the dependent step needs (null: density only).
struct NearTrial {
  const void* pts;
  int dtype;
  int32_t* lambda;  // scratch outputs of the trial
  double* delta;
};

// Default layouts (measured on the GB300): density in segments from 2 gridded
// dimensions up; the near phase in segments in 3, union otherwise.
inline int default_dlayout(int g) { return g >= 2 ? kLayoutSegment : kLayoutUnion; }
inline int default_nlayout(int g) { return g == 3 ? kLayoutSegment : kLayoutUnion; }
// segments of the segment layouts span cells while their union fits this
inline int default_seg_cells(int g) { return g == 3 ? 48 : 0; }

// The grid level and kernel layouts of one (class, cutoff): a fixed radius or
// layout from the flags, else the autotuned choice (measured now when the
// call asks for autotuning and the shape is new, cached otherwise), else the
// default rule.  A trial, per radius, times cells, then density in both
// layouts and the dependent search (near phase + far phase) with each near
// layout (after one untimed pass that loads the kernels and warms the caches);
// the radius with the least cells + best density + best dependent search wins,
// with its best layouts.  The counters are saved around the trials;
// rho_scratch (and the NearTrial outputs) receive the trials' results.
Choice choose(Workspace* w, const ClassPlan& c, const ClassView& cv, CutGeom* cuts,
              const dpc_batch* b, int cut, bool fp64, int32_t* rho_scratch, uint32_t flags,
              const NearTrial* near = nullptr) {
  Choice ch;
  ch.r = (int)((flags & DPC_FLAG_RADIUS_MASK) >> 12);
  const int forced = (int)((flags & DPC_FLAG_LAYOUT_MASK) >> 16);
  const int forced_ns = (int)((flags & DPC_FLAG_NEAR_SHIFT_MASK) >> 20);
  ch.dlay = (forced && forced != kLayoutTree) ? forced : default_dlayout(c.g);
  ch.nlay = (forced && forced != kLayoutPairs) ? forced : default_nlayout(c.g);
  ch.ns = forced_ns ? forced_ns - 1 : 0;
  ch.sc = default_seg_cells(c.g);
  const std::string key = (near ? "R/" : "D/") + tune_key(c, b, cut);
  auto it = w->tuned.find(key);
  const bool fixed = ch.r != 0 || forced || forced_ns;
  if (!fixed && it == w->tuned.end() && (flags & DPC_FLAG_AUTOTUNE)) {
    cudaStream_t st = w->stream;
    if (!w->tune_ev[0])
      for (auto& e : w->tune_ev) cudaEventCreate(&e);
    cudaMemcpyAsync(w->ctr_save, w->ctr, sizeof(Counters), cudaMemcpyDeviceToDevice, st);
    // the tensor layout exists for 5-8 dimensions with the float32 filter
    const int ndl = (c.dp == 8 && !fp64) ? 4 : 3;
    const int dlays[4] = {kLayoutUnion, kLayoutSegment, kLayoutPairs, kLayoutTensor};
    // the tensor layouts exist for 5-8 dimensions with the float32 filter
    const int nnl = (c.dp == 8 && !fp64) ? 4 : 3;
    const int nlays[4] = {kLayoutUnion, kLayoutSegment, kLayoutTree, kLayoutTensor};
    constexpr int kShifts = 3;  // near phase 0, 1 or 2 levels below the density's
    constexpr int kNL = 4;      // near layout slots per shift
    // events: 0 start, 1 after cells, 2-5 after each density layout, 6 after
    // the subtree keys; per near shift s, 7 + (kNL + 1) s after its level
    // change and cells, then one after each near layout (each followed by the
    // far search, which finishes what the near phase leaves; the tree layout,
    // which uses no cells, only at s = 0)
    auto trial = [&](int r, bool timed) {
      if (timed) cudaEventRecord(w->tune_ev[0], st);
      launch_set_radius(cv, cuts, r, st);
      launch_cells(w->scode, cv, c.g, cuts, w->hinfo, w->hkeys, w->hvals, w->hcap, st);
      if (timed) cudaEventRecord(w->tune_ev[1], st);
      for (int l = 0; l < 4; ++l) {
        if (l < ndl)
          launch_density(c.dp, c.g, fp64, dlays[l], w->spts, w->scode, w->sid, cv, cuts, w->hinfo,
                         w->hkeys, w->hvals, w->pieces, rho_scratch, w->skey, w->ctr, st,
                         default_seg_cells(c.g));
        if (timed) cudaEventRecord(w->tune_ev[2 + l], st);
      }
      if (!near) return;
      launch_tree_maxkey(w->skey, w->spts, c.dp, cv.N, w->nodes, w->leaf_parent, w->visit, w->nbox,
                         !w->boxes_ready, st);
      w->boxes_ready = true;
      if (timed) cudaEventRecord(w->tune_ev[6], st);
      for (int sh = 0; sh < kShifts; ++sh) {
        if (sh > 0) {
          launch_set_radius(cv, cuts, r, st);
          launch_near_level(cv, cuts, sh, st);
          launch_cells(w->scode, cv, c.g, cuts, w->hinfo, w->hkeys, w->hvals, w->hcap, st);
        }
        if (timed) cudaEventRecord(w->tune_ev[7 + (kNL + 1) * sh], st);
        for (int l = 0; l < kNL; ++l) {
          if (l < nnl && (sh == 0 || nlays[l] != kLayoutTree)) {
            if (nlays[l] == kLayoutTensor)
              launch_dep_near_tc(c.g, w->spts, w->sid, w->skey, cv, 0, near->pts, near->dtype,
                                 cuts, w->hinfo, w->hkeys, w->hvals, w->pieces, near->lambda,
                                 near->delta, queue_of(w), w->ctr, st);
            else
              launch_dep_near(c.dp, c.g, fp64, nlays[l], w->spts, w->scode, w->skey, cv, 0,
                              near->pts, near->dtype, cuts, w->hinfo, w->hkeys, w->hvals,
                              near->lambda, near->delta, queue_of(w), w->ctr, st,
                              default_seg_cells(c.g));
            launch_dep_far(c.dp, fp64, w->spts, w->scode, w->skey, cv, cuts, w->nodes, w->nbox,
                           w->roots, queue_of(w), near->lambda, near->delta, w->ctr, st);
          }
          if (timed) cudaEventRecord(w->tune_ev[8 + (kNL + 1) * sh + l], st);
        }
      }
    };
    auto span = [&](int a, int z) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, w->tune_ev[a], w->tune_ev[z]) != cudaSuccess) {
        cudaGetLastError();
        return 1e30f;
      }
      return ms;
    };
    const int rmax = c.g >= 4 ? 1 : (c.g == 3 ? 2 : 3);
    trial(1, false);  // untimed: module loading, caches
    Choice best;
    float best_ms = 0.f;
    bool failed = false;
    for (int r = 1; r <= rmax && !failed; ++r) {
      // each phase: the smaller of two timings
      float cl = 1e30f, dt[4] = {1e30f, 1e30f, 1e30f, 1e30f};
      float nt[kShifts][kNL], lv[kShifts];
      for (int sh = 0; sh < kShifts; ++sh) {
        lv[sh] = 1e30f;
        for (int l = 0; l < kNL; ++l) nt[sh][l] = 1e30f;
      }
      for (int rep = 0; rep < 2; ++rep) {
        trial(r, true);
        if (cudaEventSynchronize(w->tune_ev[near ? 8 + (kNL + 1) * (kShifts - 1) + kNL - 1 : 5]) !=
            cudaSuccess) {
          cudaGetLastError();
          failed = true;
          break;
        }
        cl = fminf(cl, span(0, 1));
        for (int l = 0; l < ndl; ++l) dt[l] = fminf(dt[l], span(1 + l, 2 + l));
        if (near)
          for (int sh = 0; sh < kShifts; ++sh) {
            // the level change and cells of a shift count against it
            lv[sh] = sh == 0 ? 0.f
                             : fminf(lv[sh], span(8 + (kNL + 1) * (sh - 1) + kNL - 1, 7 + (kNL + 1) * sh));
            for (int l = 0; l < nnl; ++l)
              if (sh == 0 || nlays[l] != kLayoutTree)
                nt[sh][l] = fminf(nt[sh][l], span(7 + (kNL + 1) * sh + l, 8 + (kNL + 1) * sh + l));
          }
      }
      if (failed) break;
      // a layout other than the default has to win by 3%
      auto pick = [&](const float* t, const int* lays, int m, int def) {
        int bi = 0;
        for (int l = 0; l < m; ++l)
          if (lays[l] == def) bi = l;
        for (int l = 0; l < m; ++l)
          if (t[l] < 0.97f * t[bi]) bi = l;
        return bi;
      };
      const int di = pick(dt, dlays, ndl, default_dlayout(c.g));
      int nsi = 0, ni = -1;
      float nms = 0.f;
      if (near) {
        ni = pick(nt[0], nlays, nnl, default_nlayout(c.g));
        nms = nt[0][ni];
        for (int sh = 1; sh < kShifts; ++sh) {
          const int l = pick(nt[sh], nlays, nnl, default_nlayout(c.g));
          const float t = lv[sh] + nt[sh][l];
          if (t < 0.97f * nms) {
            nms = t;
            nsi = sh;
            ni = l;
          }
        }
      }
      const float ms = cl + dt[di] + nms;
      if (best.r == 0 || ms < best_ms) {
        best_ms = ms;
        best.r = r;
        best.dlay = dlays[di];
        best.nlay = near ? nlays[ni] : default_nlayout(c.g);
        best.ns = near ? nsi : 0;
        best.sc = default_seg_cells(c.g);
      }
    }
    if (failed) best = Choice();
    // back to the default level (the trials left a shifted one behind)
    launch_set_radius(cv, cuts, 0, st);
    cudaMemcpyAsync(w->ctr, w->ctr_save, sizeof(Counters), cudaMemcpyDeviceToDevice, st);
    it = w->tuned.emplace(key, best).first;
  }
  if (!fixed && it != w->tuned.end() && it->second.r > 0) ch = it->second;
  if (ch.r > 0) launch_set_radius(cv, cuts, ch.r, w->stream);
  w->last_choice = ch;
  return ch;
}

void reset_call(Workspace* w, uint32_t flags) {
  w->begin_call(flags);
  cudaMemsetAsync(w->status, 0, sizeof(int), w->stream);
  cudaMemsetAsync(w->ctr, 0, sizeof(Counters), w->stream);
}

// Reserves the workspace for a plan and uploads its tables.
int prepare(Workspace* w, CallPlan& P, const dpc_batch* b, const std::vector<Inst>& insts,
            const dpc_params* params, uint32_t flags) {
  sort_init();
  P.params = params;
  P.skip_noise = (flags & DPC_FLAG_SKIP_NOISE) != 0;
  int rc = w->reserve(P.max_n, P.max_inst, P.ncut);
  if (rc) return rc;
  reset_call(w, flags);
  return upload_tables(w, P, b, insts, params);
}

}  // namespace
}  // namespace dpc

using namespace dpc;

extern "C" {

const char* dpc_version(void) { return "0.3.0"; }

int dpc_cut_band(double d_cut, int32_t dim, float* out) {
  if (!out || dim < 1 || dim > kMaxDim || !std::isfinite(d_cut) || d_cut < 0.0) return DPC_ERR_ARG;
  const CutHost h = make_cut_host(d_cut, dp_of(dim));
  out[0] = h.t_in;
  out[1] = h.t_out;
  out[2] = h.band_mul;
  out[3] = h.band_add;
  return DPC_OK;
}

const char* dpc_strerror(int status) {
  switch (status) {
    case DPC_OK: return "ok";
    case DPC_ERR_ARG: return "invalid argument";
    case DPC_ERR_CUDA: return "CUDA error or no CUDA device";
    case DPC_ERR_OOM: return "device memory allocation failed";
    case DPC_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case DPC_ERR_OVERFLOW: return "an instance, or the whole batch, has 2^31 or more points";
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
  if (flags & DPC_FLAG_SKIP_NOISE) return DPC_ERR_ARG;  // no thresholds here
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (N > 0 && (!pts || !rho)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  CallPlan P = make_plan(b, insts, 0, b->n_dcut, false);
  if ((rc = prepare(w, P, b, insts, nullptr, flags))) return rc;
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  for (const ClassPlan& c : P.classes) {
    const ClassView cv = view_of(w, c, insts);
    bin_class(w, pts, dtype, P, c, cv, b, insts);
    for (int k = 0; k < P.ncut; ++k) {
      CutGeom* cuts = w->cuts + (size_t)k * cv.ninst;
      const Choice ch = choose(w, c, cv, cuts, b, k, fp64, rho + (size_t)k * N, flags);
      cells_step(w, c, cv, cuts);
      density_step(w, c, cv, cuts, fp64, ch.dlay, ch.sc, rho + (size_t)k * N);
    }
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
  if (flags & DPC_FLAG_SKIP_NOISE) return DPC_ERR_ARG;  // rho_skip is the argument here
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (dcut_index < 0 || dcut_index >= b->n_dcut) return DPC_ERR_ARG;
  if (N > 0 && (!pts || !rho || !lambda || !delta)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  CallPlan P = make_plan(b, insts, dcut_index, 1, false);
  if ((rc = prepare(w, P, b, insts, nullptr, flags))) return rc;
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  for (const ClassPlan& c : P.classes) {
    const ClassView cv = view_of(w, c, insts);
    bin_class(w, pts, dtype, P, c, cv, b, insts);
    tree_step(w, cv);
    const Choice ch = choose(w, c, cv, w->cuts, b, dcut_index, fp64, nullptr,
                             flags & ~DPC_FLAG_AUTOTUNE, nullptr);
    cells_step(w, c, cv, w->cuts);
    launch_keys_from_rho(rho, w->sid, cv.N, w->skey, w->stream);
    dependent_step(w, c, cv, w->cuts, pts, dtype, rho_skip, fp64, ch.nlay, ch.ns, ch.sc, lambda,
                   delta);
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
  if (flags & ~kKnownFlags) return DPC_ERR_ARG;
  if (dcut_index < 0 || dcut_index >= b->n_dcut || !params) return DPC_ERR_ARG;
  if (N > 0 && (!rho || !lambda || !delta || !label)) return DPC_ERR_ARG;
  for (int i = 0; i < b->n_inst; ++i)
    if (std::isnan(params[(size_t)i * b->n_dcut + dcut_index].delta_min)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  CallPlan P = make_plan(b, insts, dcut_index, 1, true);
  if ((rc = prepare(w, P, b, insts, params, flags))) return rc;
  for (const ClassPlan& c : P.classes) {
    const ClassView cv = view_of(w, c, insts);
    launch_class_init(cv, c.g, c.ib, c.bcap, w->status, w->stream);
    launch_chunks(cv, w->chunk_inst, w->chunk_pos, w->stream);
    labels_step(w, c, cv, 0, one_params(params, c, P.ncut_all, dcut_index), rho, lambda, delta,
                label);
  }
  return finish(w, flags);
}

// The kernels of every class and cutoff (the part of dpc_run a graph holds).
// A phase of one cutoff finished for every class: stage 0 after the density
// (rho), 1 after the dependent search (lambda, delta), 2 after the labels.
using StageDone = std::function<void(int stage, int cut)>;

static void run_classes(Workspace* w, const CallPlan& P, const void* pts, int dtype,
                        const dpc_batch* b, const std::vector<Inst>& insts, uint64_t N,
                        const dpc_params* params, int32_t* rho, int32_t* lambda, double* delta,
                        int32_t* label, uint32_t flags, const StageDone* done = nullptr) {
  const bool fp64 = (flags & DPC_PREC_MASK) == DPC_PREC_FP64;
  for (const ClassPlan& c : P.classes) {
    // classes run one after another on the stream, so a phase of the last
    // class finishes that phase's output of every class
    const bool last = &c == &P.classes.back();
    const ClassView cv = view_of(w, c, insts);
    bin_class(w, pts, dtype, P, c, cv, b, insts);
    tree_step(w, cv);
    for (int k = 0; k < P.ncut; ++k) {
      const size_t o = (size_t)k * N;
      CutGeom* cuts = w->cuts + (size_t)k * cv.ninst;
      const NearTrial nt{pts, dtype, lambda + o, delta + o};
      const Choice ch = choose(w, c, cv, cuts, b, k, fp64, rho + o, flags, &nt);
      cells_step(w, c, cv, cuts);
      density_step(w, c, cv, cuts, fp64, ch.dlay, ch.sc, rho + o);
      if (last && done) (*done)(0, k);
      dependent_step(w, c, cv, cuts, pts, dtype, 0, fp64, ch.nlay, ch.ns, ch.sc, lambda + o,
                     delta + o);
      if (last && done) (*done)(1, k);
      labels_step(w, c, cv, k, one_params(params, c, P.ncut_all, k), rho + o, lambda + o,
                  delta + o, label + o);
      if (last && done) (*done)(2, k);
    }
  }
}

int dpc_decision_graph(const dpc_batch* b, const int32_t* rho, const double* delta, int32_t k,
                       int32_t* top, double* gamma, int32_t rho_bins, int32_t delta_bins,
                       double delta_lo, int64_t* hist, uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_batch(b, &insts, &N);
  if (rc) return rc;
  if (flags & ~(DPC_FLAG_SYNC_CHECK)) return DPC_ERR_ARG;
  if (k < 0 || k > decision_max_topk()) return DPC_ERR_ARG;
  if (rho_bins < 0 || rho_bins > 32 || delta_bins < 0 || delta_bins > 2048) return DPC_ERR_ARG;
  if ((rho_bins > 0) != (delta_bins > 0)) return DPC_ERR_ARG;
  if (k > 0 && (!top || !gamma)) return DPC_ERR_ARG;
  if (rho_bins > 0 && (!hist || !(delta_lo > 0.0) || !std::isfinite(delta_lo))) return DPC_ERR_ARG;
  if (N > 0 && (!rho || !delta)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  // every non-empty instance in one class (the summaries do not depend on the
  // dimension); rows of empty instances keep the padding written first
  CallPlan P = make_plan(b, insts, 0, 1, true);
  if ((rc = prepare(w, P, b, insts, nullptr, flags))) return rc;
  launch_decision_init(b->n_inst, k, top, gamma, rho_bins, delta_bins,
                       (unsigned long long*)hist, w->stream);
  for (const ClassPlan& c : P.classes) {
    const ClassView cv = view_of(w, c, insts);
    if (k > 0 &&
        (rc = w->reserve_buf(&w->scr, &w->scr_bytes, decision_scratch_bytes(cv.ninst, k))))
      return rc;
    launch_class_init(cv, c.g, c.ib, c.bcap, w->status, w->stream);
    launch_chunks(cv, w->chunk_inst, w->chunk_pos, w->stream);
    launch_decision(rho, delta, cv, k, top, gamma, rho_bins, delta_bins, delta_lo,
                    (unsigned long long*)hist, w->scr, w->stream);
  }
  return finish(w, flags);
}

int dpc_priority_range(const void* pts, int dtype, const dpc_batch* b, const int32_t* rho,
                       int32_t n_query, const int32_t* q_inst, const double* q_box,
                       const int32_t* q_rho, int32_t max_out, int64_t* count, int32_t* ids,
                       uint32_t flags, void* stream) {
  std::vector<Inst> insts;
  uint64_t N = 0;
  int rc = check_batch(b, &insts, &N);
  if (rc) return rc;
  if (flags & ~(DPC_FLAG_SYNC_CHECK)) return DPC_ERR_ARG;
  if (dtype != DPC_I32 && dtype != DPC_F32) return DPC_ERR_ARG;
  if (n_query < 0 || max_out < 0) return DPC_ERR_ARG;
  if (n_query == 0) return DPC_OK;
  if (!q_inst || !q_box || !q_rho || !count || (max_out > 0 && !ids)) return DPC_ERR_ARG;
  if (N > 0 && (!pts || !rho)) return DPC_ERR_ARG;
  Workspace* w = nullptr;
  if ((rc = get_workspace((cudaStream_t)stream, &w))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  // classes by dimension; the first cutoff of every instance sizes its grid
  // (the tree does not depend on it)
  CallPlan P = make_plan(b, insts, 0, 1, false);
  if ((rc = prepare(w, P, b, insts, nullptr, flags))) return rc;
  cudaStream_t st = w->stream;
  const uint32_t nq = (uint32_t)n_query;
  const size_t o_cnt = 0;
  const size_t o_off = align_up(sizeof(uint32_t) * nq);
  const size_t o_map = o_off + align_up(sizeof(unsigned long long) * (nq + 1));
  const size_t bytes = o_map + align_up(sizeof(int32_t) * (size_t)b->n_inst);
  if ((rc = w->reserve_buf(&w->scr, &w->scr_bytes, bytes))) return rc;
  uint32_t* cnt = (uint32_t*)((char*)w->scr + o_cnt);
  unsigned long long* off = (unsigned long long*)((char*)w->scr + o_off);
  int32_t* rowmap = (int32_t*)((char*)w->scr + o_map);
  PrangeArgs a;
  a.nq = nq;
  a.n_inst = b->n_inst;
  a.q_inst = q_inst;
  a.q_box = q_box;
  a.q_rho = q_rho;
  a.rowmap = nullptr;
  a.one_row = -1;
  a.count = (long long*)count;
  a.stack_cap = 0;
  if (const char* e = std::getenv("DPC_RANGE_STACK")) a.stack_cap = std::atoi(e);
  launch_prange_init(a, ids, max_out, w->status, st);
  std::vector<int32_t> map_host((size_t)b->n_inst);
  for (const ClassPlan& c : P.classes) {
    const ClassView cv = view_of(w, c, insts);
    bin_class(w, pts, dtype, P, c, cv, b, insts);
    tree_step(w, cv);
    launch_keys_from_rho(rho, w->sid, cv.N, w->skey, st);
    launch_tree_maxkey(w->skey, w->spts, c.dp, cv.N, w->nodes, w->leaf_parent, w->visit, w->nbox,
                       true, st);
    w->boxes_ready = true;
    if (c.uploaded()) {
      std::fill(map_host.begin(), map_host.end(), -1);
      for (size_t j = 0; j < c.members.size(); ++j) map_host[c.members[j]] = (int32_t)j;
      // pageable source: staged before the call returns
      cudaMemcpyAsync(rowmap, map_host.data(), sizeof(int32_t) * map_host.size(),
                      cudaMemcpyHostToDevice, st);
      a.rowmap = rowmap;
      a.one_row = -1;
    } else {
      a.rowmap = nullptr;
      a.one_row = c.members[0];
    }
    launch_prange(c.dp, false, w->spts, w->sid, w->skey, cv, w->nodes, w->nbox, w->roots, a, cnt,
                  nullptr, nullptr, w->status, st);
    if (max_out == 0) continue;
    launch_prange_scan(cnt, nq, off, st);
    unsigned long long total = 0;
    if (cudaMemcpyAsync(&total, off + nq, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    if (total == 0) continue;
    if (total >= (1ull << 32)) return DPC_ERR_OVERFLOW;
    const uint32_t tn = (uint32_t)total;
    const size_t k_a = 0;
    const size_t k_b = align_up(sizeof(unsigned long long) * tn);
    const size_t v_a = 2 * k_b;
    const size_t v_b = v_a + align_up(sizeof(uint32_t) * tn);
    const size_t h_o = v_b + align_up(sizeof(uint32_t) * tn);
    const size_t need = h_o + align_up(sizeof(uint32_t) * sort_hist_words(tn));
    if ((rc = w->reserve_buf(&w->scr2, &w->scr2_bytes, need))) return rc;
    char* s2 = (char*)w->scr2;
    unsigned long long* keys_a = (unsigned long long*)(s2 + k_a);
    unsigned long long* keys_b = (unsigned long long*)(s2 + k_b);
    launch_prange(c.dp, true, w->spts, w->sid, w->skey, cv, w->nodes, w->nbox, w->roots, a, cnt, off,
                  keys_a, w->status, st);
    // sort the keys (query << 31 | id): 31 id bits under ib query bits
    int ib = 0;
    while (ib < 32 && (1ull << ib) < nq) ++ib;
    ClassGeom g;
    std::memset(&g, 0, sizeof(g));
    g.S = 31;
    g.ib = ib;
    g.status = w->status;
    cudaMemcpyAsync(w->cls, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    launch_sort(keys_a, keys_b, (uint32_t*)(s2 + v_a), (uint32_t*)(s2 + v_b), tn, w->cls,
                (uint32_t*)(s2 + h_o), st);
    const int passes = sort_passes(31, ib);
    launch_prange_scatter((passes & 1) ? keys_b : keys_a, total, off, nq, max_out, ids, w->status, st);
  }
  return finish(w, flags);
}

static int run_device(Workspace* w, const void* pts, int dtype, const dpc_batch* b,
                      const std::vector<Inst>& insts, uint64_t N, const dpc_params* params,
                      int32_t* rho, int32_t* lambda, double* delta, int32_t* label,
                      uint32_t flags, const StageDone* done = nullptr) {
  CallPlan P = make_plan(b, insts, 0, b->n_dcut, false);
  int rc = prepare(w, P, b, insts, params, flags);
  if (rc) return rc;
  run_classes(w, P, pts, dtype, b, insts, N, params, rho, lambda, delta, label, flags, done);
  return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}

// Everything a captured graph depends on: the pointers, the batch, the
// thresholds and the flags that change the kernel sequence.
static std::string graph_key(const void* pts, int dtype, const dpc_batch* b,
                             const dpc_params* params, const void* rho, const void* lambda,
                             const void* delta, const void* label, uint32_t flags) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  const void* ptrs[5] = {pts, rho, lambda, delta, label};
  put(ptrs, sizeof(ptrs));
  const uint32_t f = flags & (DPC_PREC_MASK | DPC_FLAG_RADIUS_MASK | DPC_FLAG_LAYOUT_MASK);
  put(&dtype, sizeof(dtype));
  put(&f, sizeof(f));
  put(&b->n_inst, sizeof(b->n_inst));
  put(&b->n_dcut, sizeof(b->n_dcut));
  put(b->pt_offset, sizeof(int64_t) * (b->n_inst + 1));
  put(b->dim, sizeof(int32_t) * b->n_inst);
  if (b->coord_offset) put(b->coord_offset, sizeof(int64_t) * b->n_inst);
  put(b->d_cut, sizeof(double) * b->n_inst * b->n_dcut);
  put(params, sizeof(dpc_params) * b->n_inst * b->n_dcut);
  return k;
}

// dpc_run with DPC_FLAG_GRAPH: the kernels of a call are captured into a CUDA
// graph on the first call with a new key and replayed afterwards.  The
// per-call work outside the graph: status reset and the instance tables' copy.
static int run_graph(Workspace* w, const void* pts, int dtype, const dpc_batch* b,
                     const std::vector<Inst>& insts, uint64_t N, const dpc_params* params,
                     int32_t* rho, int32_t* lambda, double* delta, int32_t* label, uint32_t flags) {
  if (w->stream == nullptr) return DPC_ERR_UNSUPPORTED;  // the legacy stream cannot be captured
  const uint32_t f = flags & ~(DPC_FLAG_PHASE_TIMES | DPC_FLAG_AUTOTUNE);
  CallPlan P = make_plan(b, insts, 0, b->n_dcut, false);
  int rc = prepare(w, P, b, insts, params, f);
  if (rc) return rc;
  std::string key = graph_key(pts, dtype, b, params, rho, lambda, delta, label, f);
  if (!w->gexec || key != w->gkey) {
    w->drop_graph();
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(w->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    const long long before = g_kernel_launches;
    run_classes(w, P, pts, dtype, b, insts, N, params, rho, lambda, delta, label, f);
    const cudaError_t e1 = cudaStreamEndCapture(w->stream, &g);
    if (e1 != cudaSuccess || g == nullptr) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return DPC_ERR_CUDA;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&w->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      w->gexec = nullptr;
      return DPC_ERR_CUDA;
    }
    w->gkey.swap(key);
    w->glaunches = g_kernel_launches - before;
  } else {
    g_kernel_launches += w->glaunches;
  }
  if (cudaGraphLaunch(w->gexec, w->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPC_ERR_CUDA;
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
  if (flags & DPC_FLAG_GRAPH)
    rc = run_graph(w, pts, dtype, b, insts, N, params, rho, lambda, delta, label, flags);
  else
    rc = run_device(w, pts, dtype, b, insts, N, params, rho, lambda, delta, label, flags);
  if (rc) return rc;
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
  // each output goes back as soon as its phase has finished (a copy stream
  // behind an event), overlapping the phases still to run
  if (!w->copy_stream && cudaStreamCreateWithFlags(&w->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    w->copy_stream = nullptr;
    return DPC_ERR_CUDA;
  }
  const size_t nev = 3u * (size_t)b->n_dcut;
  while (w->out_ev.size() < nev) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return DPC_ERR_CUDA;
    }
    w->out_ev.push_back(e);
  }
  cudaStream_t cs = w->copy_stream;
  const StageDone done = [&](int stage, int k) {
    const size_t o = (size_t)k * N;
    cudaEvent_t ev = w->out_ev[3u * (size_t)k + (size_t)stage];
    cudaEventRecord(ev, st);
    cudaStreamWaitEvent(cs, ev, 0);
    if (N == 0) return;
    if (stage == 0) {
      cudaMemcpyAsync(rho_host + o, io + o_rho + 4 * o, 4 * N, cudaMemcpyDeviceToHost, cs);
    } else if (stage == 1) {
      cudaMemcpyAsync(lambda_host + o, io + o_lam + 4 * o, 4 * N, cudaMemcpyDeviceToHost, cs);
      cudaMemcpyAsync(delta_host + o, io + o_del + 8 * o, 8 * N, cudaMemcpyDeviceToHost, cs);
    } else {
      cudaMemcpyAsync(label_host + o, io + o_lab + 4 * o, 4 * N, cudaMemcpyDeviceToHost, cs);
    }
  };
  if (elems) cudaMemcpyAsync(io + o_pts, pts_host, 4 * elems, cudaMemcpyHostToDevice, st);
  rc = run_device(w, io + o_pts, dtype, b, insts, N, params, (int32_t*)(io + o_rho),
                  (int32_t*)(io + o_lam), (double*)(io + o_del), (int32_t*)(io + o_lab), flags,
                  &done);
  // no copy into the caller's buffers may outlive the call, whatever happened
  const cudaError_t ec = cudaStreamSynchronize(cs);
  if (rc) return rc;
  if (ec != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
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
  cudaMemcpy(&c, w->ctr, sizeof(c), cudaMemcpyDeviceToHost);
  out->band_pairs = (int64_t)c.band_pairs;
  out->far_queries = (int64_t)c.far_queries;
  out->exact_rescans = (int64_t)c.exact_rescans;
  out->kernel_launches = w->launches_last;
  out->far_nodes = (int64_t)c.far_nodes;
  out->far_nodes_max = (int64_t)c.far_nodes_max;
  out->density_pairs = (int64_t)c.pairs;
  if (w->have_last) {
    CutGeom cg;
    GridGeom g;
    HashInfo hi;
    cudaMemcpy(&cg, w->last_cut, sizeof(cg), cudaMemcpyDeviceToHost);
    cudaMemcpy(&g, w->last_geom, sizeof(g), cudaMemcpyDeviceToHost);
    cudaMemcpy(&hi, w->hinfo, sizeof(hi), cudaMemcpyDeviceToHost);
    out->occupied_cells = hi.m;
    out->grid_level = cg.k;
    out->block_radius = cg.R;
    out->density_layout = w->last_choice.dlay;
    out->near_layout = w->last_choice.nlay;
    out->near_shift = w->last_choice.ns;
    out->bits_per_axis = g.B;
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
