/*
 * dpc.h -- C ABI of the GB300 exact Density Peaks Clustering library.
 *
 * What is computed (Huang, Yu, Shun, "Faster Parallel Exact Density Peaks
 * Clustering", Section 3):
 *   rho_i     Definition 1: the number of points j with D(x_i, x_j) <= d_cut,
 *             the point itself included.
 *   lambda_i  Definition 2: the nearest point of strictly higher density;
 *             density ties are broken by id (the smaller id is higher), distance
 *             ties go to the smaller id.  -1 for the highest point.
 *   delta_i   Definition 3: D(x_i, lambda_i); +inf for the highest point.
 *   label_i   Definitions 4-5 and the assignment rule after them: noise
 *             (rho < rho_noise) gets -1; a center (not noise, and either no
 *             dependent point or rho >= rho_min and delta >= delta_min) gets its
 *             own id; every other point gets its dependent point's label.
 *
 * Distances are exact: int32 inputs use the exact integer squared distance;
 * float32 inputs use the binary64 value
 *     s = (((t_0*t_0) + t_1*t_1) + ...),  t_k = (double)x_ik - (double)x_jk,
 * each operation rounded to nearest, no fused multiply-add.  The density
 * predicate is s <= fl64(d_cut*d_cut); delta = sqrt(s) rounded to nearest.
 * The fast paths filter in float32 with a proven error band and re-evaluate
 * every undecided pair in binary64, so all outputs are identical to that
 * definition whatever precision mode is chosen.
 *
 * Conventions shared by every entry point:
 *   - Points are row-major [n][d], d in 1..8, int32 or float32.  int32
 *     coordinates must satisfy |x| <= 2^24, float32 ones must be finite with
 *     |x| <= 2^60 (so every squared distance is exact in binary64 for integers
 *     and representable in float32); otherwise the call fails with
 *     DPC_ERR_DATA (reported when DPC_FLAG_SYNC_CHECK is set, or by
 *     dpc_last_status).
 *   - Ids are 0-based and local to each instance of a batch.
 *   - Unless stated otherwise pointers to points and results are DEVICE
 *     pointers owned by the caller; the library never frees them.  The
 *     library owns an internal workspace per (device, stream), grown on
 *     demand with cudaMalloc and freed by dpc_release().  The first call at a
 *     given size therefore allocates; later calls of the same or smaller size
 *     do not.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Calls on different streams use
 *     different workspaces and may overlap.
 *   - Return value: DPC_OK or a negative dpc_status.  Argument errors are
 *     detected on the host before any work is queued; nothing is written to
 *     the outputs then.  Errors found on the device (bad coordinates, a
 *     bounded wait that expired) are recorded in a per-workspace status word:
 *     with DPC_FLAG_SYNC_CHECK the call synchronizes the stream and returns
 *     that status; otherwise dpc_last_status() returns it later.
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     entry point returns DPC_ERR_CUDA.
 *   - Every wait inside a kernel (the radix sort's look-back over earlier
 *     tiles, the tensor-core density's wait for its MMA) is bounded; when the
 *     bound runs out the kernel records DPC_ERR_TIMEOUT and finishes.  The
 *     sort then counts the earlier tiles' digits itself, so its result stays
 *     exact; the tensor-core density leaves the pieces it did not finish at
 *     density 0.  Either way no later kernel reads or writes out of bounds.
 *   - Environment variables, read at every call:
 *       DPC_WORKSPACE_LIMIT_BYTES  the largest single device allocation the
 *         library may make; a call that needs more fails with DPC_ERR_OOM
 *         before any work is queued (unset: no limit).
 *       DPC_TEST_WAIT_LIMIT  for tests: polls before a bounded wait gives up
 *         (only lowers the built-in limit; 0 makes every such wait give up at
 *         once).  A call captured with DPC_FLAG_GRAPH keeps the value it was
 *         captured with.
 */
#ifndef DPC_H
#define DPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DPC_OK = 0,
  DPC_ERR_ARG = -1,         /* invalid argument (detected on the host)         */
  DPC_ERR_CUDA = -2,        /* a CUDA call failed or no device is available    */
  DPC_ERR_OOM = -3,         /* workspace allocation failed                     */
  DPC_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up              */
  DPC_ERR_OVERFLOW = -5,    /* an instance, or the whole batch, has 2^31 or
                               more points                                     */
  DPC_ERR_UNSUPPORTED = -6, /* valid request this build does not implement     */
  DPC_ERR_DATA = -7         /* coordinates out of the supported range / NaN, or
                               dependent pointers that do not form a forest    */
} dpc_status;

/* coordinate types */
enum { DPC_I32 = 0, DPC_F32 = 1 };

/* precision modes (flags & DPC_PREC_MASK).  Both give identical results. */
enum {
  DPC_PREC_FP64 = 0,     /* every distance evaluated in binary64              */
  DPC_PREC_FP32_CERT = 1 /* float32 filter + binary64 recheck of the band     */
};
#define DPC_PREC_MASK 0xFu
#define DPC_FLAG_SYNC_CHECK (1u << 8)  /* synchronize and return the device status */
#define DPC_FLAG_PHASE_TIMES (1u << 9) /* record CUDA events around every phase
                                          (read with dpc_get_phase_times)      */
/* Autotune the grid level and the kernel layouts: the first dpc_run /
 * dpc_density call that sees a new (dimension class, instance count, point
 * count, cutoff) shape runs, once per candidate block radius (R = 1, 2, 3 for
 * d <= 2; R = 1, 2 for d = 3; d >= 4 has R = 1 only; the cells shrink as R
 * grows), the cell-hash step, the density kernel in every density layout and
 * (for dpc_run) the near-dependent and far search for every near layout at
 * 0, 1 and 2 grid levels below the density's, timing each with CUDA events
 * and synchronizing the stream, and keeps the fastest for that shape in the
 * workspace; later calls (with or without the flag) reuse the choice without
 * synchronizing.  Results do not depend on the choice.  Do not set it on a
 * call that is being captured into a CUDA graph. */
#define DPC_FLAG_AUTOTUNE (1u << 10)
/* Fixed block radius r = 1..5 instead of the default rule or the autotuned
 * choice (larger radii are clamped to the largest the dimension allows: 5 for
 * d <= 2, 2 for d = 3, 1 for d >= 4).  Results do not depend on it. */
#define DPC_FLAG_RADIUS(r) ((uint32_t)(r) << 12)
#define DPC_FLAG_RADIUS_MASK (0x7u << 12)
/* Fixed work layout of the density and near-dependent kernels instead of the
 * default rule (density in segments for d >= 2; the near phase in segments for
 * d = 3, union otherwise) or the autotuned choice:
 * 1 = union (a warp's 32 consecutive points, one query per lane, the union of
 * their blocks streamed as broadcast reads), 2 = segment (the block of one
 * cell spread over the lanes, the cell's queries one at a time), 3 = tree
 * (near phase only, density keeps its default: no block scan, every query goes
 * to the tree search of the far phase), 4 = tensor (density and near phase,
 * 5-8 dimensions with DPC_PREC_FP32_CERT: distance tiles on the tensor cores
 * with a certified error band; other cases use segment for the density and
 * union for the near phase), 5 = pairs (density only:
 * the segment layout evaluating every unordered pair once and counting it for
 * both points), 6 = cell (density and near phase: one warp per occupied cell,
 * the cell's block staged in shared memory, every lane one query -- or a share
 * of one query's candidates in cells of fewer than 32 points -- against all of
 * it).  Results do not depend on it. */
#define DPC_FLAG_LAYOUT(v) ((uint32_t)(v) << 16)
#define DPC_FLAG_LAYOUT_MASK (0x7u << 16)
/* dpc_run only: capture the call's kernels into a CUDA graph the first time a
 * (pointers, batch, thresholds, precision, radius) combination is seen, and on
 * later calls with the same combination launch that graph instead of one
 * kernel at a time.  Each call still resets the status word and copies the
 * instance tables (outside the graph), so the point coordinates may change
 * between calls; a different combination, or a workspace that had to grow,
 * captures anew.  Needs a stream other than the legacy default stream
 * (DPC_ERR_UNSUPPORTED there).  Phase times are not recorded and autotuning is
 * not done in this mode (autotune with a call without the flag first). */
#define DPC_FLAG_GRAPH (1u << 11)
/* dpc_run / dpc_run_host only: skip the dependent-point search of the noise
 * points, as Algorithm 1 queries only the points at or above the density
 * threshold.  A point of instance i with rho < rho_noise of (i, cutoff) gets
 * lambda = -1 and delta = NaN; it is noise, so its label is -1 either way.
 * Every other output is unchanged: the points a non-noise point can depend on
 * are denser than it, hence never noise. */
#define DPC_FLAG_SKIP_NOISE (1u << 15)
/* Fixed grid level of the near-dependent phase: DPC_FLAG_NEAR_SHIFT(j), j =
 * 0..2, searches the (2R+1)^g block of cells j levels finer than the density
 * step's (a block 2^j times narrower: fewer candidates per query, more queries
 * left to the tree search); without it the default (j = 0) or the autotuned
 * choice.  Results do not depend on it. */
#define DPC_FLAG_NEAR_SHIFT(j) (((uint32_t)(j) + 1u) << 20)
#define DPC_FLAG_NEAR_SHIFT_MASK (0x3u << 20)

/* A batch of independent point sets packed back to back.  n_inst = 1 for a
 * single point set.  All arrays are HOST arrays read during the call only. */
typedef struct {
  int32_t n_inst;
  const int64_t* pt_offset;    /* [n_inst+1]: instance i owns points
                                  [pt_offset[i], pt_offset[i+1]) of the packed
                                  result arrays; pt_offset[0] = 0              */
  const int64_t* coord_offset; /* [n_inst]: element offset of instance i's
                                  first coordinate in `pts`; NULL means
                                  pt_offset[i] * dim[i]                        */
  const int32_t* dim;          /* [n_inst]: d of each instance, 1..8           */
  int32_t n_dcut;              /* cutoffs per instance (a sweep), >= 1         */
  const double* d_cut;         /* [n_inst * n_dcut], finite and >= 0; entry
                                  i*n_dcut + k is cutoff k of instance i       */
} dpc_batch;

/* Labelling thresholds of one (instance, cutoff) pair (Definitions 4-5). */
typedef struct {
  int32_t rho_noise; /* rho < rho_noise -> noise                               */
  int32_t rho_min;   /* centers need rho >= rho_min ...                        */
  double delta_min;  /* ... and delta >= delta_min                             */
} dpc_params;

/* Densities (Definition 1) for every cutoff of every instance.
 *   pts   device, packed coordinates (see dpc_batch), int32 or float32 (dtype)
 *   rho   device, int32 [n_dcut][N], N = pt_offset[n_inst]; rho[k*N + p] is
 *         the density of packed point p under that instance's cutoff k. */
int dpc_density(const void* pts, int dtype, const dpc_batch* b, int32_t* rho, uint32_t flags,
                void* stream);

/* Dependent points and distances (Definitions 2-3) for cutoff `dcut_index`,
 * given the densities of that cutoff.
 *   rho       device, int32 [N], as written by dpc_density for that cutoff
 *   rho_skip  points with rho < rho_skip are skipped (lambda -1, delta NaN),
 *             as the paper skips noise points (Algorithm 1); 0 = none
 *   lambda    device, int32 [N], instance-local id of the dependent point or -1
 *   delta     device, double [N]; +inf for the highest point of an instance
 * The cutoff is used only to size the search grid; the results depend on
 * (pts, rho) alone. */
int dpc_dependent(const void* pts, int dtype, const dpc_batch* b, int32_t dcut_index,
                  const int32_t* rho, int32_t rho_skip, int32_t* lambda, double* delta,
                  uint32_t flags, void* stream);

/* Labels (Definitions 4-5 and the assignment rule) for cutoff `dcut_index`.
 *   params  host, [n_inst * n_dcut] thresholds (entry i*n_dcut + dcut_index is
 *           used for instance i)
 *   rho, lambda, delta  device, [N], as produced by the two calls above
 *   label   device, int32 [N]: instance-local id of the cluster center, or -1
 * lambda must form a forest within each instance (as dpc_dependent writes
 * it); a pointer that has not reached a root (a center or a noise point)
 * after the fixed number of pointer-jumping rounds (enough for any forest)
 * reveals a cycle, reported as DPC_ERR_DATA. */
int dpc_cluster(const dpc_batch* b, int32_t dcut_index, const dpc_params* params,
                const int32_t* rho, const int32_t* lambda, const double* delta, int32_t* label,
                uint32_t flags, void* stream);

/* Decision-graph summaries of one cutoff's (rho, delta) arrays (Section 3:
 * d_cut, rho_min and delta_min are picked from the graph of delta against
 * rho).  Two products per instance, both computed on the device:
 *   top, gamma  device, int32 / double [n_inst][k]: the k points with the
 *               largest gamma = fl64(rho * delta) -- the center score of
 *               Rodriguez and Laio, unrelated to the priority value of the
 *               priority search kd-tree -- in descending gamma, equal gamma
 *               by the smaller instance-local id; the top point's gamma is
 *               +inf.  Points whose product is NaN (delta NaN: a point
 *               skipped with rho_skip) or negative take no part.  Rows of
 *               instances with fewer than k such points end in (-1, NaN).
 *               k in [0, 1024]; k = 0 skips this product (top, gamma unused).
 *   hist        device, int64 [n_inst][rho_bins][delta_bins]: counts of the
 *               points with rho >= 1 and a non-NaN delta by
 *                 rho bin   = floor(log2 rho)
 *                 delta bin = 0 if delta <= delta_lo, else the binary
 *                             exponent of fl64(delta / delta_lo)
 *               each clipped to its last bin (+inf delta lands in the last
 *               delta bin).  rho_bins in [0, 32], delta_bins in [0, 2048],
 *               both 0 (skip, hist unused) or both positive; delta_lo finite
 *               and > 0 when used.
 *   rho, delta  device, [N] for one cutoff (slices of dpc_run's outputs or
 *               what dpc_density / dpc_dependent wrote).
 * Only the point counts and offsets of `b` are read; its coordinates and
 * cutoffs are not.  Flags: DPC_FLAG_SYNC_CHECK only.  All outputs are
 * written in stream order; a bad argument returns DPC_ERR_ARG with nothing
 * launched. */
int dpc_decision_graph(const dpc_batch* b, const int32_t* rho, const double* delta, int32_t k,
                       int32_t* top, double* gamma, int32_t rho_bins, int32_t delta_bins,
                       double delta_lo, int64_t* hist, uint32_t flags, void* stream);

/* Priority range search (the appendix on range queries of the priority
 * search kd-tree): for each query, the points of one instance inside a closed
 * axis-parallel box whose priority -- the density rho -- is above a
 * threshold:  { i : lo[a] <= x_i[a] <= hi[a] for a < d, and rho_i > rho_q }.
 * The search runs on the same radix tree as the dependent-point step,
 * entering a subtree only if its largest density is above rho_q and its
 * bounding box meets the query box.
 *   pts, dtype, b  the points, as for dpc_density (the first cutoff of every
 *                  instance sizes the search grid; results do not depend on it)
 *   rho       device, int32 [N]: the priorities (normally one cutoff's rho)
 *   n_query   number of queries (0: nothing is done)
 *   q_inst    device, int32 [n_query]: the batch row of each query's instance
 *   q_box     device, double [n_query][2][8]: lo[0..7] then hi[0..7]; only
 *             the first dim[q_inst] entries of each are read; coordinates are
 *             compared exactly (a NaN bound matches nothing)
 *   q_rho     device, int32 [n_query]: the thresholds rho_q
 *   count     device, int64 [n_query]: number of matching points
 *   ids       device, int32 [n_query][max_out]: the min(count, max_out)
 *             smallest matching instance-local ids, ascending, then -1;
 *             max_out = 0 computes the counts only (ids unused)
 * A q_inst outside [0, n_inst) leaves count 0 and sets the device status
 * (DPC_ERR_DATA with DPC_FLAG_SYNC_CHECK).  With max_out > 0 the call reads
 * the number of matches back once per dimension class, so it synchronizes
 * `stream`; more than 2^32 - 1 matches in one class returns DPC_ERR_OVERFLOW.
 * Flags: DPC_FLAG_SYNC_CHECK only.  The environment variable
 * DPC_RANGE_STACK (1..2048) caps the per-warp node stack; a smaller cap sends
 * more subtrees to the per-lane walk (for testing that path; results do not
 * depend on it). */
int dpc_priority_range(const void* pts, int dtype, const dpc_batch* b, const int32_t* rho,
                       int32_t n_query, const int32_t* q_inst, const double* q_box,
                       const int32_t* q_rho, int32_t max_out, int64_t* count, int32_t* ids,
                       uint32_t flags, void* stream);

/* The whole pipeline for every cutoff: one binning per instance, then for each
 * cutoff density, dependent points and labels.  The instances of a batch are
 * processed together in at most five groups of equal padded dimension and
 * gridded axes (d = 1; d = 2; d = 3; d = 4; d = 5..8), each kernel launched
 * once per group, so the launch count does not grow with the number of
 * instances.
 *   params                   host, [n_inst * n_dcut] thresholds
 *   rho, lambda, delta, label  device, [n_dcut][N] each (cutoff-major) */
int dpc_run(const void* pts, int dtype, const dpc_batch* b, const dpc_params* params,
            int32_t* rho, int32_t* lambda, double* delta, int32_t* label, uint32_t flags,
            void* stream);

/* dpc_run on HOST buffers: copies the points to the device, runs, copies the
 * four results back and synchronizes `stream` before returning.  Each result
 * is copied back on a stream the library owns as soon as the phase that
 * writes it has finished (rho after the density, lambda and delta after the
 * dependent search, the labels last), overlapping the phases still to run;
 * every copy has finished when the call returns, also on error.  Host buffers
 * that are page-locked copy faster (and only those overlap).  Same layouts as
 * dpc_run. */
int dpc_run_host(const void* pts_host, int dtype, const dpc_batch* b, const dpc_params* params,
                 int32_t* rho_host, int32_t* lambda_host, double* delta_host,
                 int32_t* label_host, uint32_t flags, void* stream);

/* dpc_density for ONE point set without allocating device memory.  The paper
 * has no counterpart.  It is for callers that cannot let a library call
 * cudaMalloc: a host application that hands out all device memory through its
 * own allocator or budget (an allocation behind its back can fail or push it
 * over that budget), and latency-critical paths, where cudaMalloc and cudaFree
 * may synchronize the device.
 *   pts     device, [n][d] row-major, int32 or float32 (dtype), same range
 *           rules as every other entry point
 *   n       0 .. DPC_STATIC_MAX_POINTS; larger n fails with DPC_ERR_OVERFLOW
 *           before any work is queued
 *   d       1..8; d_cut finite and >= 0
 *   rho     device, int32 [n]: the same densities dpc_density writes for this
 *           point set and cutoff
 *   flags   precision (DPC_PREC_*) and DPC_FLAG_SYNC_CHECK as for dpc_density
 * All scratch memory is one fixed array of about 7 MB compiled into the
 * library, so every GPU that loads the library holds it until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The call never allocates (no cudaMalloc,
 * cudaFree or allocating library routine) and issues only kernels and
 * memsets on `stream`; it clears the words that must start at zero itself.
 * All calls share the one array, which keeps the last call's contents: calls
 * that overlap on the GPU (on different streams, or from several threads
 * without ordering) race and corrupt each other's results; order them on one
 * stream. */
#define DPC_STATIC_MAX_POINTS 65536
int dpc_density_static(const void* pts, int dtype, int64_t n, int32_t d, double d_cut,
                       int32_t* rho, uint32_t flags, void* stream);

/* Counters from the last call on `stream` (synchronizes the stream). */
typedef struct {
  int64_t band_pairs;     /* density pairs re-evaluated in binary64          */
  int64_t far_queries;    /* dependent queries not settled by the grid block */
  int64_t exact_rescans;  /* dependent queries whose float32 winner was
                             ambiguous and were re-ranked in binary64        */
  int64_t occupied_cells; /* occupied grid cells of the last cutoff          */
  int32_t grid_level;     /* level of the density grid of the last cutoff    */
  int32_t bits_per_axis;  /* Morton bits per gridded axis of the last binning */
  int64_t kernel_launches;/* kernels the last call enqueued                  */
  int64_t far_nodes;      /* radix-tree nodes expanded by the far queries    */
  int64_t far_nodes_max;  /* most nodes expanded by a single far query       */
  int32_t block_radius;   /* block radius R of the last cutoff (cells per side
                             of the (2R+1)^g block around a query's cell)     */
  int32_t density_layout; /* layout the last density launch ran: 1 union,
                             2 segment, 4 tensor, 5 pairs, 6 cell
                             (see DPC_FLAG_LAYOUT)                            */
  int32_t near_layout;    /* layout of the last near-dependent launch: 1 union,
                             2 segment, 3 tree, 4 tensor, 6 cell              */
  int32_t near_shift;     /* grid levels the near phase ran below the density's */
  int64_t density_pairs;  /* (query, candidate) pairs the density step scanned
                             (every cutoff and instance of the last call)    */
} dpc_stats;
int dpc_get_stats(void* stream, dpc_stats* out);

/* Phases of a call, for DPC_FLAG_PHASE_TIMES. */
enum {
  DPC_PHASE_BIN = 0,      /* bbox, grid setup, Morton codes, radix sort, gather */
  DPC_PHASE_TREE = 1,     /* radix tree over the sorted points                 */
  DPC_PHASE_CELLS = 2,    /* occupied cells of the density level + hash        */
  DPC_PHASE_DENSITY = 3,  /* the density kernel (one launch per cutoff)        */
  DPC_PHASE_MAXKEY = 4,   /* subtree maximum keys                              */
  DPC_PHASE_NEAR = 5,     /* dependent points, grid-block phase (one launch)   */
  DPC_PHASE_FAR = 6,      /* dependent points, tree phase (one launch)         */
  DPC_PHASE_LABELS = 7,   /* labels                                            */
  DPC_NUM_PHASES = 8
};
/* Milliseconds spent in each phase by the last call on `stream` that set
 * DPC_FLAG_PHASE_TIMES, summed over its instances and cutoffs, measured with
 * CUDA events on that stream; launches[p] is the number of times phase p ran.
 * Synchronizes the stream. */
typedef struct {
  double ms[DPC_NUM_PHASES];
  int64_t launches[DPC_NUM_PHASES];
} dpc_phase_times;
int dpc_get_phase_times(void* stream, dpc_phase_times* out);

/* Device-side status of the last call on `stream` (synchronizes it). */
int dpc_last_status(void* stream);

/* The float32 certification band of one cutoff.  Host arithmetic only (no
 * device is touched), so it can be checked without a GPU.  A float32 squared
 * distance s32 evaluated the way the density and dependent kernels do it
 * (t_k = x_ik - x_jk rounded to float32, s32 = fmaf(t_k, t_k, s32) over the
 * coordinates in increasing k, from s32 = 0) and the canonical binary64 value
 * s64 of the same pair satisfy
 *     s32 <= t_in   =>  s64 <= fl64(d_cut * d_cut)
 *     s32 >  t_out  =>  s64 >  fl64(d_cut * d_cut)
 * and, for two pairs a and b from the same query,
 *     s32_b > s32_a * band_mul + band_add  =>  s64_b > s64_a,
 * for float32 coordinates whose squares stay in the normal float32 range
 * (the entry points' |x| <= 2^60 rule).  Pairs between t_in and t_out are
 * recounted in binary64; ambiguous dependent candidates are re-ranked in
 * binary64.  The bound is the standard one for a sum of m = dp + 2 rounded
 * operations (gamma_m = m u / (1 - m u), u = 2^-24 and 2^-53, dp = 2, 4 or 8
 * the padded dimension of `dim`), rounded outwards to float32.
 *   dim  1..8
 *   out  host, float[4]: t_in, t_out, band_mul, band_add
 * Returns DPC_OK, or DPC_ERR_ARG for a bad dim, a negative or non-finite
 * d_cut, or a NULL out. */
int dpc_cut_band(double d_cut, int32_t dim, float* out);

/* Measured arithmetic peak of this GPU, for the rooflines of the distance
 * kernels; the paper has no counterpart.  kind 0: float32 fused multiply-add
 * (FFMA), kind 1: binary64 (DFMA).  *flops_per_s = 2 flops per FMA x the FMAs
 * of a multiply-add loop (8 independent chains per thread, 4 CTAs of 512
 * threads per SM) / the median time of 5 launches timed with CUDA events on
 * `stream`, at whatever clocks the GPU runs (nothing is changed).
 * Synchronizes the stream; allocates and frees a buffer of 8 KB per SM.
 * Returns DPC_OK, DPC_ERR_ARG (bad kind or NULL), DPC_ERR_OOM or
 * DPC_ERR_CUDA. */
int dpc_probe_peak(int kind, double* flops_per_s, void* stream);

/* Short description of a status code (static storage). */
const char* dpc_strerror(int status);

/* Library version, e.g. "0.1.0". */
const char* dpc_version(void);

/* Free every workspace of every device and stream.  Must not overlap with
 * running calls. */
void dpc_release(void);

#ifdef __cplusplus
}
#endif

#endif /* DPC_H */
