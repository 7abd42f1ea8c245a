/*
 * dpc_oracle_tree.c -- exact Density Peaks Clustering for large point sets,
 * on the CPU, with a priority search kd-tree.
 *
 * TEST INFRASTRUCTURE ONLY.  Like dpc_oracle.c this is part of the checker
 * the CUDA library is compared with: only the test suite, the smoke check and
 * the CPU baseline leg of the benchmark may load it.  It shares no code with
 * the library, nor with dpc_oracle.c (the brute-force definitions it is
 * itself checked against); the three agree only through the specification.
 *
 * What it computes is exactly what dpc_oracle.c computes -- Definitions 1-3
 * of Section 3 under the same fixed readings (R1-R5 there):
 *   rho_i    = #{j : s_ij <= fl64(d_cut^2)}, the point itself included;
 *   lambda_i = the least (s_ij, j) over the points j higher than i, where j is
 *              higher iff rho_j > rho_i, or rho_j == rho_i and j < i;
 *   delta_i  = sqrt(s_i,lambda_i), +inf for the highest point; points with
 *              rho_i < rho_skip get lambda = -1, delta = NaN;
 *   s_ij     = the exact int64 squared distance for int32 points, and for
 *              float32 points the binary64 sum (((t_0^2) + t_1^2) + ...) of
 *              t_k = (double)x_ik - (double)x_jk in increasing k, each
 *              operation rounded to nearest, no fused multiply-add.
 * How it gets there follows the paper's own exact algorithm rather than the
 * O(n^2) definition: a kd-tree over the points whose every node keeps its
 * bounding box and the highest point below it (the priority search kd-tree
 * of Section 4.1), a fixed-radius count on that tree for rho (Section 6.1:
 * a subtree entirely inside the ball is counted whole) and, for lambda, the
 * priority nearest-neighbour search of Algorithm 1: visit nearer subtrees
 * first, skip a subtree whose highest point is not higher than the query or
 * whose box is farther than the best candidate found so far.
 *
 * Why the pruning is exact, with no safety margin.  The box bound of a node
 * is computed with the very operations of s_ij, each term replaced by the
 * gap between the query and the box on that axis (0 inside the box's span):
 * rounding to nearest is monotone and symmetric, so for every point of the
 * box |fl(q_k - x_k)| >= |fl(q_k - lo_k)| (or hi_k), squares and then partial
 * sums taken in the same order keep that order, and the computed bound is
 * <= the computed s of every point in the box.  Likewise the far-corner
 * bound is >= the computed s of every point in it.  Hence a node whose lower
 * bound exceeds fl64(d_cut^2) holds no neighbour, a node whose upper bound
 * does not exceed it holds only neighbours, and a node whose lower bound
 * exceeds the best s so far holds no better candidate -- including ties,
 * because equality is not pruned.  For int32 points all of this is exact
 * integer arithmetic.
 *
 * The tree splits every node with more than kLeaf points at the median of
 * its widest axis (so its depth is about log2(n / kLeaf)); a node whose box
 * is a single point (all duplicates) is a leaf of any size.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { T_I32 = 0, T_F32 = 1 };
enum { kLeaf = 64, kMaxDimT = 8, kMaxCuts = 32 };

/* ---- one point set in tree order ---------------------------------------- */

typedef struct {
  int32_t left, right; /* children, -1 for a leaf */
  int64_t begin, end;  /* the node's points: positions [begin, end) */
} tnode;

typedef struct {
  int dtype;
  int d;
  int64_t n;
  int64_t* id;   /* tree position -> original index */
  double* xf;    /* float points: [n][d] coordinates in tree order (exact) */
  int32_t* xi;   /* int points: [n][d] coordinates in tree order */
  tnode* node;
  double* box;   /* [nodes][2][d]: lo then hi per node */
  int32_t nodes;
  int32_t cap;   /* nodes allocated */
} ktree;

static double coord(const ktree* T, int64_t p, int k) {
  return T->dtype == T_I32 ? (double)T->xi[p * T->d + k] : T->xf[p * T->d + k];
}

/* swap two positions of the tree order */
static void swap_pos(ktree* T, int64_t a, int64_t b) {
  int64_t t = T->id[a];
  T->id[a] = T->id[b];
  T->id[b] = t;
  for (int k = 0; k < T->d; ++k) {
    if (T->dtype == T_I32) {
      int32_t u = T->xi[a * T->d + k];
      T->xi[a * T->d + k] = T->xi[b * T->d + k];
      T->xi[b * T->d + k] = u;
    } else {
      double u = T->xf[a * T->d + k];
      T->xf[a * T->d + k] = T->xf[b * T->d + k];
      T->xf[b * T->d + k] = u;
    }
  }
}

/* Rearrange positions [lo, hi) so that position m holds the value of rank
   m - lo on axis k, smaller-or-equal values before it and larger-or-equal
   after it (quickselect with a three-way partition, so runs of equal values
   cost linear time). */
static void select_median(ktree* T, int64_t lo, int64_t hi, int64_t m, int k, uint64_t* rng) {
  while (hi - lo > 1) {
    *rng = *rng * 6364136223846793005ull + 1442695040888963407ull;
    int64_t pv = lo + (int64_t)((*rng >> 33) % (uint64_t)(hi - lo));
    double pivot = coord(T, pv, k);
    /* [lo, lt) < pivot, [lt, i) == pivot, [gt, hi) > pivot */
    int64_t lt = lo, i = lo, gt = hi;
    while (i < gt) {
      double v = coord(T, i, k);
      if (v < pivot) {
        swap_pos(T, lt, i);
        ++lt;
        ++i;
      } else if (v > pivot) {
        --gt;
        swap_pos(T, i, gt);
      } else {
        ++i;
      }
    }
    if (m < lt)
      hi = lt;
    else if (m >= gt)
      lo = gt;
    else
      return;
  }
}

static void node_box(ktree* T, int32_t v) {
  double* lo = T->box + (size_t)v * 2 * T->d;
  double* hi = lo + T->d;
  const tnode* nd = &T->node[v];
  for (int k = 0; k < T->d; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (int64_t p = nd->begin; p < nd->end; ++p)
    for (int k = 0; k < T->d; ++k) {
      double c = coord(T, p, k);
      if (c < lo[k]) lo[k] = c;
      if (c > hi[k]) hi[k] = c;
    }
}

/* Nodes are numbered in preorder, so every child has a larger number than
   its parent. */
static int32_t build_node(ktree* T, int64_t begin, int64_t end, uint64_t* rng) {
  if (T->nodes >= T->cap) return -1; /* cannot happen: see tree_build */
  int32_t v = T->nodes++;
  T->node[v].begin = begin;
  T->node[v].end = end;
  T->node[v].left = T->node[v].right = -1;
  node_box(T, v);
  if (end - begin <= kLeaf) return v;
  const double* lo = T->box + (size_t)v * 2 * T->d;
  const double* hi = lo + T->d;
  int axis = 0;
  double wide = -1.0;
  for (int k = 0; k < T->d; ++k)
    if (hi[k] - lo[k] > wide) {
      wide = hi[k] - lo[k];
      axis = k;
    }
  if (!(wide > 0.0)) return v; /* every point of the node is the same point */
  int64_t mid = begin + (end - begin) / 2;
  select_median(T, begin, end, mid, axis, rng);
  int32_t l = build_node(T, begin, mid, rng);
  int32_t r = build_node(T, mid, end, rng);
  if (l < 0 || r < 0) return -1;
  T->node[v].left = l;
  T->node[v].right = r;
  return v;
}

static int tree_build(ktree* T, const void* pts, int dtype, int64_t n, int d) {
  memset(T, 0, sizeof(*T));
  T->dtype = dtype;
  T->d = d;
  T->n = n;
  /* a split node has more than kLeaf points and halves them, so every leaf
     but a lone root holds at least kLeaf / 2 points: at most n / 4 + 1
     leaves and twice as many nodes */
  int64_t cap = 2 * (n / (kLeaf / 2) + 1) + 1;
  if (cap > INT32_MAX) return -1;
  T->cap = (int32_t)cap;
  T->id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  T->node = (tnode*)malloc(sizeof(tnode) * (size_t)cap);
  T->box = (double*)malloc(sizeof(double) * 2 * (size_t)d * (size_t)cap);
  if (dtype == T_I32)
    T->xi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1) * (size_t)d);
  else
    T->xf = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1) * (size_t)d);
  if (!T->id || !T->node || !T->box || (!T->xi && !T->xf)) return -1;
  for (int64_t i = 0; i < n; ++i) {
    T->id[i] = i;
    for (int k = 0; k < d; ++k) {
      if (dtype == T_I32)
        T->xi[i * d + k] = ((const int32_t*)pts)[i * d + k];
      else
        T->xf[i * d + k] = (double)((const float*)pts)[i * d + k];
    }
  }
  if (n > 0) {
    uint64_t rng = 0x9e3779b97f4a7c15ull;
    if (build_node(T, 0, n, &rng) < 0) return -1;
  }
  return 0;
}

static void tree_free(ktree* T) {
  free(T->id);
  free(T->node);
  free(T->box);
  free(T->xi);
  free(T->xf);
  memset(T, 0, sizeof(*T));
}

/* ---- the squared distance and its box bounds ----------------------------- */

/* float points: s of positions p and q (R1, binary64, fixed order) */
static double sq_f(const ktree* T, int64_t p, int64_t q) {
  const double* a = T->xf + p * T->d;
  const double* b = T->xf + q * T->d;
  double s = 0.0;
  for (int k = 0; k < T->d; ++k) {
    double t = a[k] - b[k];
    double t2 = t * t;
    s = s + t2;
  }
  return s;
}

static int64_t sq_i(const ktree* T, int64_t p, int64_t q) {
  const int32_t* a = T->xi + p * T->d;
  const int32_t* b = T->xi + q * T->d;
  int64_t s = 0;
  for (int k = 0; k < T->d; ++k) {
    int64_t t = (int64_t)a[k] - (int64_t)b[k];
    s += t * t;
  }
  return s;
}

/* lower and upper bounds of s over the points of node v, query position p */
static void bounds_f(const ktree* T, int64_t p, int32_t v, double* lb, double* ub) {
  const double* q = T->xf + p * T->d;
  const double* lo = T->box + (size_t)v * 2 * T->d;
  const double* hi = lo + T->d;
  double sl = 0.0, su = 0.0;
  for (int k = 0; k < T->d; ++k) {
    double g = 0.0;
    if (q[k] < lo[k])
      g = q[k] - lo[k];
    else if (q[k] > hi[k])
      g = q[k] - hi[k];
    double g2 = g * g;
    sl = sl + g2;
    double f1 = q[k] - lo[k], f2 = q[k] - hi[k];
    double f = fabs(f1) > fabs(f2) ? f1 : f2;
    double f2sq = f * f;
    su = su + f2sq;
  }
  *lb = sl;
  *ub = su;
}

static void bounds_i(const ktree* T, int64_t p, int32_t v, int64_t* lb, int64_t* ub) {
  const int32_t* q = T->xi + p * T->d;
  const double* lo = T->box + (size_t)v * 2 * T->d;
  const double* hi = lo + T->d;
  int64_t sl = 0, su = 0;
  for (int k = 0; k < T->d; ++k) {
    int64_t x = q[k], l = (int64_t)lo[k], h = (int64_t)hi[k];
    int64_t g = x < l ? l - x : (x > h ? x - h : 0);
    sl += g * g;
    int64_t f1 = x > l ? x - l : l - x, f2 = x > h ? x - h : h - x;
    int64_t f = f1 > f2 ? f1 : f2;
    su += f * f;
  }
  *lb = sl;
  *ub = su;
}

/* ---- density: all cutoffs in one walk ------------------------------------ */

/* The cutoffs in increasing order of fl64(d_cut^2) (ties keep their input
   order); out[r] is the input index of rank r. */
typedef struct {
  int ncut;
  int out[kMaxCuts];
  double dc2[kMaxCuts];   /* fl64(d_cut^2), ascending */
  int64_t dc2i[kMaxCuts]; /* its floor, the same predicate on exact integers */
} cutset;

static void make_cutset(cutset* C, int ncut, const double* d_cut) {
  C->ncut = ncut;
  for (int c = 0; c < ncut; ++c) {
    double v = d_cut[c] * d_cut[c];
    int r = c;
    while (r > 0 && C->dc2[r - 1] > v) { /* insertion sort, stable */
      C->dc2[r] = C->dc2[r - 1];
      C->out[r] = C->out[r - 1];
      --r;
    }
    C->dc2[r] = v;
    C->out[r] = c;
  }
  for (int r = 0; r < ncut; ++r)
    C->dc2i[r] = C->dc2[r] >= 9.0e18 ? INT64_MAX : (int64_t)floor(C->dc2[r]);
}

/* first rank r in [a, b) whose cutoff admits a squared distance s (b if none) */
static int first_rank_f(const cutset* C, int a, int b, double s) {
  while (a < b && s > C->dc2[a]) ++a;
  return a;
}

static int first_rank_i(const cutset* C, int a, int b, int64_t s) {
  while (a < b && s > C->dc2i[a]) ++a;
  return a;
}

typedef struct {
  int32_t v;
  int16_t a, b; /* ranks [a, b) still undecided for this subtree */
} dstack_item;

/* counts[c] = rho of the point at position p for every cutoff c (input
   order).  Ranks are counted through a difference array: a neighbour, or a
   whole subtree, first admitted at rank r adds to every rank from r up to the
   end of the range still open for it. */
static void density_query(const ktree* T, const cutset* C, int64_t p, int64_t* counts,
                          dstack_item* stack) {
  int64_t diff[kMaxCuts + 1];
  for (int r = 0; r <= C->ncut; ++r) diff[r] = 0;
  int top = 0;
  if (T->n > 0) {
    stack[top].v = 0;
    stack[top].a = 0;
    stack[top].b = (int16_t)C->ncut;
    ++top;
  }
  while (top > 0) {
    dstack_item it = stack[--top];
    const tnode* nd = &T->node[it.v];
    int a, w; /* ranks below a: nobody within; ranks >= w: everybody */
    if (T->dtype == T_I32) {
      int64_t lb, ub;
      bounds_i(T, p, it.v, &lb, &ub);
      a = first_rank_i(C, it.a, it.b, lb);
      w = first_rank_i(C, a, it.b, ub);
    } else {
      double lb, ub;
      bounds_f(T, p, it.v, &lb, &ub);
      a = first_rank_f(C, it.a, it.b, lb);
      w = first_rank_f(C, a, it.b, ub);
    }
    if (w < it.b) { /* the whole subtree is within every rank in [w, b) */
      diff[w] += nd->end - nd->begin;
      diff[it.b] -= nd->end - nd->begin;
    }
    if (a >= w) continue; /* nothing left open */
    if (nd->left < 0) {
      for (int64_t q = nd->begin; q < nd->end; ++q) {
        int r = T->dtype == T_I32 ? first_rank_i(C, a, w, sq_i(T, p, q))
                                  : first_rank_f(C, a, w, sq_f(T, p, q));
        diff[r] += 1;
        diff[w] -= 1;
      }
      continue;
    }
    stack[top].v = nd->left;
    stack[top].a = (int16_t)a;
    stack[top].b = (int16_t)w;
    ++top;
    stack[top].v = nd->right;
    stack[top].a = (int16_t)a;
    stack[top].b = (int16_t)w;
    ++top;
  }
  int64_t run = 0;
  for (int r = 0; r < C->ncut; ++r) {
    run += diff[r];
    counts[C->out[r]] = run;
  }
}

/* ---- dependent point: Algorithm 1's priority nearest-neighbour search ---- */

/* order key: a larger key is higher in the total order (R3) */
static uint64_t order_key(int32_t rho, int64_t id) {
  return ((uint64_t)(uint32_t)rho << 32) | (uint64_t)(0xffffffffu - (uint32_t)id);
}

/* maxkey[v] = the largest order key among the points of node v; children
   have larger node numbers, so one reverse sweep computes it */
static void node_maxkeys(const ktree* T, const int32_t* rho_by_id, uint64_t* maxkey) {
  for (int32_t v = T->nodes - 1; v >= 0; --v) {
    const tnode* nd = &T->node[v];
    uint64_t m = 0;
    if (nd->left < 0) {
      for (int64_t q = nd->begin; q < nd->end; ++q) {
        uint64_t k = order_key(rho_by_id[T->id[q]], T->id[q]);
        if (k > m) m = k;
      }
    } else {
      m = maxkey[nd->left] > maxkey[nd->right] ? maxkey[nd->left] : maxkey[nd->right];
    }
    maxkey[v] = m;
  }
}

typedef struct {
  int32_t v;
  double lbf;
  int64_t lbi;
} nstack_item;

/* lambda (original id, -1 if none) and delta of the point at position p */
static void dependent_query(const ktree* T, const int32_t* rho_by_id, const uint64_t* maxkey,
                            int64_t p, int64_t* lam, double* delta, nstack_item* stack) {
  const int64_t me = T->id[p];
  const uint64_t kme = order_key(rho_by_id[me], me);
  int64_t best = -1;       /* original id */
  double bestf = INFINITY; /* float points */
  int64_t besti = INT64_MAX;
  int top = 0;
  stack[top].v = 0;
  stack[top].lbf = 0.0;
  stack[top].lbi = 0;
  ++top;
  while (top > 0) {
    nstack_item it = stack[--top];
    if (maxkey[it.v] <= kme) continue; /* no point below is higher than the query */
    if (best >= 0) {
      if (T->dtype == T_I32 ? it.lbi > besti : it.lbf > bestf) continue; /* too far */
    }
    const tnode* nd = &T->node[it.v];
    if (nd->left < 0) {
      for (int64_t q = nd->begin; q < nd->end; ++q) {
        int64_t j = T->id[q];
        if (order_key(rho_by_id[j], j) <= kme) continue;
        if (T->dtype == T_I32) {
          int64_t s = sq_i(T, p, q);
          if (best < 0 || s < besti || (s == besti && j < best)) {
            best = j;
            besti = s;
          }
        } else {
          double s = sq_f(T, p, q);
          if (best < 0 || s < bestf || (s == bestf && j < best)) {
            best = j;
            bestf = s;
          }
        }
      }
      continue;
    }
    /* push the farther child first so that the nearer one is searched first */
    nstack_item a, b;
    a.v = nd->left;
    b.v = nd->right;
    double u;
    if (T->dtype == T_I32) {
      int64_t ui;
      bounds_i(T, p, a.v, &a.lbi, &ui);
      bounds_i(T, p, b.v, &b.lbi, &ui);
      a.lbf = b.lbf = 0.0;
      if (a.lbi < b.lbi) {
        nstack_item t = a;
        a = b;
        b = t;
      }
    } else {
      bounds_f(T, p, a.v, &a.lbf, &u);
      bounds_f(T, p, b.v, &b.lbf, &u);
      a.lbi = b.lbi = 0;
      if (a.lbf < b.lbf) {
        nstack_item t = a;
        a = b;
        b = t;
      }
    }
    stack[top++] = a; /* farther */
    stack[top++] = b; /* nearer, popped next */
  }
  *lam = best;
  if (best < 0)
    *delta = INFINITY;
  else
    *delta = T->dtype == T_I32 ? sqrt((double)besti) : sqrt(bestf);
}

/* ---- a small thread pool: parallel for over [0, m) in chunks ------------- */

typedef struct {
  void (*fn)(void* ctx, int64_t begin, int64_t end, int worker);
  void* ctx;
  int64_t m, chunk;
  atomic_llong next;
  atomic_int worker_ids;
} pool_job;

static void* pool_worker(void* arg) {
  pool_job* J = (pool_job*)arg;
  int w = atomic_fetch_add(&J->worker_ids, 1);
  for (;;) {
    int64_t b = atomic_fetch_add(&J->next, J->chunk);
    if (b >= J->m) break;
    int64_t e = b + J->chunk < J->m ? b + J->chunk : J->m;
    J->fn(J->ctx, b, e, w);
  }
  return NULL;
}

static int threads_of(int threads) {
  if (threads > 0) return threads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void pool_run(int64_t m, int64_t chunk, int nt, void (*fn)(void*, int64_t, int64_t, int),
                     void* ctx) {
  pool_job J;
  J.fn = fn;
  J.ctx = ctx;
  J.m = m;
  J.chunk = chunk > 0 ? chunk : 1;
  atomic_init(&J.next, 0);
  atomic_init(&J.worker_ids, 0);
  if (nt <= 1) {
    pool_worker(&J);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
  for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, pool_worker, &J);
  for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  free(th);
}

/* ---- one point set, threads over its queries -------------------------------- */

typedef struct {
  const ktree* T;
  cutset C;
  int ncut;
  int64_t N;            /* row stride of the [ncut][N] outputs */
  int32_t* rho;         /* [ncut][N], original order */
  const int32_t* rho_c; /* one cutoff's row (dependent phase) */
  const uint64_t* maxkey;
  int32_t rho_skip;
  int32_t* lam;         /* one cutoff's row */
  double* delta;
  int64_t max_stack;
} set_job;

static void density_chunk(void* ctx, int64_t b, int64_t e, int worker) {
  (void)worker;
  set_job* J = (set_job*)ctx;
  dstack_item* stack = (dstack_item*)malloc(sizeof(dstack_item) * (size_t)J->max_stack);
  int64_t counts[kMaxCuts];
  for (int64_t p = b; p < e; ++p) {
    density_query(J->T, &J->C, p, counts, stack);
    int64_t id = J->T->id[p];
    for (int c = 0; c < J->ncut; ++c) J->rho[(size_t)c * J->N + id] = (int32_t)counts[c];
  }
  free(stack);
}

static void dependent_chunk(void* ctx, int64_t b, int64_t e, int worker) {
  (void)worker;
  set_job* J = (set_job*)ctx;
  nstack_item* stack = (nstack_item*)malloc(sizeof(nstack_item) * (size_t)J->max_stack);
  for (int64_t p = b; p < e; ++p) {
    int64_t id = J->T->id[p];
    if (J->rho_c[id] < J->rho_skip) {
      J->lam[id] = -1;
      J->delta[id] = NAN;
      continue;
    }
    int64_t lam;
    double dl;
    dependent_query(J->T, J->rho_c, J->maxkey, p, &lam, &dl, stack);
    J->lam[id] = (int32_t)lam;
    J->delta[id] = dl;
  }
  free(stack);
}

static int64_t tree_depth(const ktree* T, int32_t v) {
  if (T->node[v].left < 0) return 1;
  int64_t a = tree_depth(T, T->node[v].left), b = tree_depth(T, T->node[v].right);
  return 1 + (a > b ? a : b);
}

/* Runs one point set entirely, with `nt` threads over its queries when
   nt > 1.  Outputs are [ncut][N] rows starting at the given pointers (N is
   the row stride).  lam/delta may be NULL (density only). */
static int run_set(const void* pts, int dtype, int64_t n, int d, int ncut, const double* d_cut,
                   int32_t rho_skip, int nt, int64_t N, int32_t* rho, int32_t* lam, double* delta) {
  if (n == 0) return 0;
  ktree T;
  if (tree_build(&T, pts, dtype, n, d)) {
    tree_free(&T);
    return -3;
  }
  set_job J;
  memset(&J, 0, sizeof(J));
  J.T = &T;
  make_cutset(&J.C, ncut, d_cut);
  J.ncut = ncut;
  J.N = N;
  J.rho = rho;
  J.rho_skip = rho_skip;
  /* a DFS stack holds at most one sibling per level plus the node itself */
  J.max_stack = 2 * tree_depth(&T, 0) + 4;
  const int64_t chunk = 256;
  pool_run(n, chunk, nt, density_chunk, &J);
  if (lam && delta) {
    uint64_t* maxkey = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)T.nodes);
    if (!maxkey) {
      tree_free(&T);
      return -3;
    }
    for (int c = 0; c < ncut; ++c) {
      J.rho_c = rho + (size_t)c * N;
      node_maxkeys(&T, J.rho_c, maxkey);
      J.maxkey = maxkey;
      J.lam = lam + (size_t)c * N;
      J.delta = delta + (size_t)c * N;
      pool_run(n, chunk, nt, dependent_chunk, &J);
    }
    free(maxkey);
  }
  tree_free(&T);
  return 0;
}

/* ---- exported ---------------------------------------------------------------- */

/* One point set of n points, ncut cutoffs: rho [ncut][n]; lambda, delta
   [ncut][n] (both NULL: density only).  threads = 0: all cores. */
int orc_tree_run(const void* pts, int dtype, int64_t n, int d, int ncut, const double* d_cut,
                 int32_t rho_skip, int threads, int32_t* rho, int32_t* lambda, double* delta) {
  if (!pts || n < 0 || d < 1 || d > kMaxDimT || ncut < 1 || ncut > kMaxCuts || !d_cut || !rho)
    return -1;
  if ((lambda == NULL) != (delta == NULL)) return -1;
  return run_set(pts, dtype, n, d, ncut, d_cut, rho_skip, threads_of(threads), n, rho, lambda, delta);
}

typedef struct {
  const void* pts;
  int dtype;
  const int64_t* pt_offset;
  const int64_t* coord_offset;
  const int32_t* dim;
  const int64_t* order; /* instances, largest first */
  int ncut;
  const double* d_cut;  /* [n_inst][ncut] */
  int32_t rho_skip;
  int64_t N;
  int32_t* rho;
  int32_t* lam;
  double* delta;
  atomic_int rc;
} batch_job;

static void batch_chunk(void* ctx, int64_t b, int64_t e, int worker) {
  (void)worker;
  batch_job* J = (batch_job*)ctx;
  for (int64_t t = b; t < e; ++t) {
    int64_t i = J->order[t];
    int64_t n = J->pt_offset[i + 1] - J->pt_offset[i];
    int64_t o = J->pt_offset[i];
    const void* p = J->dtype == T_I32 ? (const void*)((const int32_t*)J->pts + J->coord_offset[i])
                                      : (const void*)((const float*)J->pts + J->coord_offset[i]);
    int rc = run_set(p, J->dtype, n, J->dim[i], J->ncut, J->d_cut + (size_t)i * J->ncut, J->rho_skip,
                     1, J->N, J->rho + o, J->lam ? J->lam + o : NULL, J->delta ? J->delta + o : NULL);
    if (rc) atomic_store(&J->rc, rc);
  }
}

static int cmp_desc_size(const void* a, const void* b);

/* A batch of n_inst independent point sets packed back to back, each with
   its own dimension and ncut cutoffs: outputs [ncut][N] with
   N = pt_offset[n_inst], instance-local ids in lambda.  One thread per
   instance, largest instances first. */
int orc_tree_batch(const void* pts, int dtype, int32_t n_inst, const int64_t* pt_offset,
                   const int64_t* coord_offset, const int32_t* dim, int ncut, const double* d_cut,
                   int32_t rho_skip, int threads, int32_t* rho, int32_t* lambda, double* delta) {
  if (!pts || n_inst < 1 || !pt_offset || !coord_offset || !dim || ncut < 1 || ncut > kMaxCuts ||
      !d_cut || !rho)
    return -1;
  if ((lambda == NULL) != (delta == NULL)) return -1;
  for (int32_t i = 0; i < n_inst; ++i)
    if (dim[i] < 1 || dim[i] > kMaxDimT || pt_offset[i + 1] < pt_offset[i]) return -1;
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_inst);
  if (!order) return -3;
  /* largest first, equal sizes by index: sort (size, index) pairs */
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)n_inst);
  if (!key) {
    free(order);
    return -3;
  }
  for (int32_t i = 0; i < n_inst; ++i) {
    key[2 * i] = pt_offset[i + 1] - pt_offset[i];
    key[2 * i + 1] = i;
  }
  qsort(key, (size_t)n_inst, 2 * sizeof(int64_t), cmp_desc_size);
  for (int32_t i = 0; i < n_inst; ++i) order[i] = key[2 * i + 1];
  free(key);
  batch_job J;
  J.pts = pts;
  J.dtype = dtype;
  J.pt_offset = pt_offset;
  J.coord_offset = coord_offset;
  J.dim = dim;
  J.order = order;
  J.ncut = ncut;
  J.d_cut = d_cut;
  J.rho_skip = rho_skip;
  J.N = pt_offset[n_inst];
  J.rho = rho;
  J.lam = lambda;
  J.delta = delta;
  atomic_init(&J.rc, 0);
  pool_run(n_inst, 1, threads_of(threads), batch_chunk, &J);
  free(order);
  return atomic_load(&J.rc);
}

static int cmp_desc_size(const void* a, const void* b) {
  const int64_t* x = (const int64_t*)a;
  const int64_t* y = (const int64_t*)b;
  if (x[0] != y[0]) return x[0] > y[0] ? -1 : 1;
  return x[1] < y[1] ? -1 : (x[1] > y[1]);
}
