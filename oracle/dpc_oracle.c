/*
 * dpc_oracle.c -- plain CPU evaluation of exact Density Peaks Clustering.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library
 * is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library never does, and the
 * two share no code.
 *
 * Everything here is the definition written out, O(n^2) where the definition
 * is O(n^2):
 *   - density          Definition 1 (Section 3): rho_i = |{j : D(x_i,x_j) <= d_cut}|,
 *                      the point itself included.
 *   - dependent point  Definitions 2-3 (Section 3): the nearest point of higher
 *                      density, with delta = its distance, +inf for the
 *                      highest point.
 *   - labels           Definitions 4-5 (Section 3) and the cluster assignment
 *                      rule that follows them.
 *
 * Fixed readings (where the paper is silent), shared with the library by
 * specification only:
 *   R1 distance: int32 input -> s = sum_k (int64)(x_ik - x_jk)^2, exact.
 *      float32 input -> s = (((t_0*t_0) + t_1*t_1) + ...) in IEEE binary64,
 *      t_k = (double)x_ik - (double)x_jk, k in increasing order, every
 *      operation rounded to nearest even, no fused multiply-add (build with
 *      -ffp-contract=off).
 *   R2 the density boundary is inclusive and compares squared values:
 *      s <= fl64(d_cut * d_cut).
 *   R3 total order: j is higher than i iff rho_j > rho_i, or rho_j == rho_i
 *      and j < i ("ties broken lexicographically", Section 3, read through the
 *      stable descending sort of Algorithm 2).
 *   R4 lambda_i = argmin over higher j of (s_ij, j): distance ties go to the
 *      smaller id, as write-min with ids does (Section 3.2, Algorithm 2).
 *   R5 delta_i = sqrt(s) correctly rounded in binary64; no higher point ->
 *      lambda = -1, delta = +inf (Definition 3); rho_i < rho_skip -> lambda = -1,
 *      delta = NaN (the noise skip of Algorithm 1).
 *   R6 noise: rho < rho_noise.  center: not noise and either lambda == -1
 *      (the highest point, or a skipped one) or rho >= rho_min and
 *      delta >= delta_min.  Every other point takes its dependent point's
 *      label; a center's label is its own index; noise gets -1.
 *
 * The `variant` bit masks below plant deliberate deviations from those
 * readings.  They exist so that tests can show each pin catches a plausible
 * mistake; variant 0 is the oracle.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { ORC_I32 = 0, ORC_F32 = 1 };

/* planted deviations (tests only) */
enum {
  ORC_VAR_EXCLUSIVE = 1,        /* s <  dc2 instead of s <= dc2           */
  ORC_VAR_NO_SELF = 2,          /* do not count the point itself          */
  ORC_VAR_TIE_LARGER_ID = 4,    /* rho ties: larger id is higher          */
  ORC_VAR_DIST_TIE_LARGER = 8,  /* distance ties: larger id wins          */
  ORC_VAR_SQRT_COMPARE = 16,    /* sqrt(s) <= d_cut instead of s <= dc2   */
  ORC_VAR_DROP_LAST_DIM = 32,   /* distance ignores the last coordinate   */
  ORC_VAR_CENTER_NO_RHO_MIN = 64 /* labels: centers skip rho >= rho_min   */
};

typedef struct {
  const void* pts;
  int dtype;
  int64_t n;
  int d;
  int variant;
} pointset;

/* ---- R1: the canonical squared distance ------------------------------- */

/* exact int64 squared distance of int32 points */
static int64_t sq_i64(const pointset* P, int64_t i, int64_t j) {
  const int32_t* x = (const int32_t*)P->pts;
  int dd = (P->variant & ORC_VAR_DROP_LAST_DIM) ? P->d - 1 : P->d;
  int64_t s = 0;
  for (int k = 0; k < dd; ++k) {
    int64_t t = (int64_t)x[i * P->d + k] - (int64_t)x[j * P->d + k];
    s += t * t;
  }
  return s;
}

/* binary64 squared distance of float32 points, fixed operation order */
static double sq_f64(const pointset* P, int64_t i, int64_t j) {
  const float* x = (const float*)P->pts;
  int dd = (P->variant & ORC_VAR_DROP_LAST_DIM) ? P->d - 1 : P->d;
  double s = 0.0;
  for (int k = 0; k < dd; ++k) {
    double t = (double)x[i * P->d + k] - (double)x[j * P->d + k];
    double t2 = t * t;
    s = s + t2;
  }
  return s;
}

/* A squared distance carried in both forms: integer inputs compare the exact
   int64, float inputs the binary64 value; delta is always sqrt of `sf`. */
typedef struct {
  int64_t si;
  double sf;
} sqd;

static sqd sqdist(const pointset* P, int64_t i, int64_t j) {
  sqd r;
  if (P->dtype == ORC_I32) {
    r.si = sq_i64(P, i, j);
    r.sf = (double)r.si;
  } else {
    r.si = 0;
    r.sf = sq_f64(P, i, j);
  }
  return r;
}

/* (a.s, ja) < (b.s, jb) in the lexicographic order of R4 */
static int sqd_less(const pointset* P, sqd a, int64_t ja, sqd b, int64_t jb) {
  if (P->dtype == ORC_I32) {
    if (a.si != b.si) return a.si < b.si;
  } else {
    if (a.sf != b.sf) return a.sf < b.sf;
  }
  if (P->variant & ORC_VAR_DIST_TIE_LARGER) return ja > jb;
  return ja < jb;
}

static double sqd_value(sqd a) { return a.sf; }

/* ---- R2: the density predicate D(x_i, x_j) <= d_cut -------------------- */

typedef struct {
  double dc;   /* d_cut as given           */
  double dc2;  /* fl64(d_cut * d_cut)      */
  int64_t dc2_int; /* floor(dc2), clamped: the same predicate on exact ints */
} cutoff;

static cutoff make_cutoff(double d_cut) {
  cutoff c;
  c.dc = d_cut;
  c.dc2 = d_cut * d_cut;
  if (c.dc2 >= 9.0e18)
    c.dc2_int = INT64_MAX;
  else
    c.dc2_int = (int64_t)floor(c.dc2);
  return c;
}

static int within(const pointset* P, const cutoff* c, sqd s) {
  if (P->variant & ORC_VAR_SQRT_COMPARE) {
    double dist = sqrt(sqd_value(s));
    if (P->variant & ORC_VAR_EXCLUSIVE) return dist < c->dc;
    return dist <= c->dc;
  }
  if (P->dtype == ORC_I32) {
    if (P->variant & ORC_VAR_EXCLUSIVE) return (double)s.si < c->dc2;
    return s.si <= c->dc2_int;
  }
  if (P->variant & ORC_VAR_EXCLUSIVE) return s.sf < c->dc2;
  return s.sf <= c->dc2;
}

/* Definition 1 for one point: count j in P with D(x_i, x_j) <= d_cut */
static int32_t density_one(const pointset* P, const cutoff* c, int64_t i) {
  int64_t count = 0;
  for (int64_t j = 0; j < P->n; ++j) {
    if (j == i && (P->variant & ORC_VAR_NO_SELF)) continue;
    if (within(P, c, sqdist(P, i, j))) ++count;
  }
  return (int32_t)count;
}

/* ---- R3: the total order ------------------------------------------------ */

/* 1 iff point j is higher than point i */
static int higher(const pointset* P, int32_t rho_j, int64_t j, int32_t rho_i, int64_t i) {
  if (rho_j != rho_i) return rho_j > rho_i;
  if (P->variant & ORC_VAR_TIE_LARGER_ID) return j > i;
  return j < i;
}

/* ---- a minimal thread pool: parallel for over [0, m) ------------------- */

typedef struct {
  void (*fn)(void* ctx, int64_t t);
  void* ctx;
  int64_t m;
  int64_t next;
  pthread_mutex_t lock;
} pfor_state;

static void* pfor_worker(void* arg) {
  pfor_state* st = (pfor_state*)arg;
  for (;;) {
    pthread_mutex_lock(&st->lock);
    int64_t t = st->next++;
    pthread_mutex_unlock(&st->lock);
    if (t >= st->m) break;
    st->fn(st->ctx, t);
  }
  return NULL;
}

static int resolve_threads(int threads) {
  if (threads > 0) return threads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void parallel_for(int64_t m, int threads, void (*fn)(void*, int64_t), void* ctx) {
  int nt = resolve_threads(threads);
  if (nt > m) nt = (int)(m > 0 ? m : 1);
  pfor_state st;
  st.fn = fn;
  st.ctx = ctx;
  st.m = m;
  st.next = 0;
  pthread_mutex_init(&st.lock, NULL);
  if (nt <= 1) {
    pfor_worker(&st);
  } else {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, pfor_worker, &st);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    free(th);
  }
  pthread_mutex_destroy(&st.lock);
}

/* ---- exported: density --------------------------------------------------- */

typedef struct {
  pointset P;
  cutoff c;
  const int64_t* idx;
  int32_t* out;
} density_job;

static void density_task(void* ctx, int64_t t) {
  density_job* J = (density_job*)ctx;
  int64_t i = J->idx ? J->idx[t] : t;
  J->out[t] = density_one(&J->P, &J->c, i);
}

/* rho for the m points idx[0..m) (all n points when idx == NULL, m == n). */
int orc_density(const void* pts, int dtype, int64_t n, int d, double d_cut,
                const int64_t* idx, int64_t m, int variant, int threads, int32_t* rho_out) {
  if (!pts || n < 0 || d < 1 || !rho_out || m < 0) return -1;
  density_job J;
  J.P.pts = pts;
  J.P.dtype = dtype;
  J.P.n = n;
  J.P.d = d;
  J.P.variant = variant;
  J.c = make_cutoff(d_cut);
  J.idx = idx;
  J.out = rho_out;
  parallel_for(idx ? m : n, threads, density_task, &J);
  return 0;
}

/* ---- exported: dependent point from a full rho array --------------------- */

typedef struct {
  pointset P;
  const int32_t* rho;
  int32_t rho_skip;
  int32_t* lam;
  double* delta;
} dependent_job;

/* Definitions 2-3 for one point: scan every point, keep the higher ones,
   take the least (s, j). */
static void dependent_task(void* ctx, int64_t i) {
  dependent_job* J = (dependent_job*)ctx;
  const pointset* P = &J->P;
  if (J->rho[i] < J->rho_skip) {
    J->lam[i] = -1;
    J->delta[i] = NAN;
    return;
  }
  int64_t best = -1;
  sqd bs;
  bs.si = 0;
  bs.sf = 0.0;
  for (int64_t j = 0; j < P->n; ++j) {
    if (!higher(P, J->rho[j], j, J->rho[i], i)) continue;
    sqd s = sqdist(P, i, j);
    if (best < 0 || sqd_less(P, s, j, bs, best)) {
      best = j;
      bs = s;
    }
  }
  J->lam[i] = (int32_t)best;
  J->delta[i] = best < 0 ? INFINITY : sqrt(sqd_value(bs));
}

int orc_dependent(const void* pts, int dtype, int64_t n, int d, const int32_t* rho,
                  int32_t rho_skip, int variant, int threads, int32_t* lambda_out,
                  double* delta_out) {
  if (!pts || n < 0 || d < 1 || !rho || !lambda_out || !delta_out) return -1;
  dependent_job J;
  J.P.pts = pts;
  J.P.dtype = dtype;
  J.P.n = n;
  J.P.d = d;
  J.P.variant = variant;
  J.rho = rho;
  J.rho_skip = rho_skip;
  J.lam = lambda_out;
  J.delta = delta_out;
  parallel_for(n, threads, dependent_task, &J);
  return 0;
}

/* ---- exported: dependent point of selected points, rho computed on demand --
 *
 * For a query i, walk the other points in increasing (s_ij, j) order -- each
 * step is a full scan for the least pair above the previous one -- and stop at
 * the first point whose density (Definition 1, computed from scratch) makes it
 * higher than i.  That point is lambda_i by Definition 2 read with R3/R4.
 * Needs no density array, so it works on point sets far too large for the
 * O(n^2) routines.  Stops after `max_checks` candidates and reports the query
 * as unresolved (status 0); status 1 = resolved, lambda/delta written.
 */
typedef struct {
  pointset P;
  cutoff c;
  const int64_t* idx;
  int64_t max_checks;
  int32_t* lam;
  double* delta;
  int32_t* rho_q;
  int8_t* status;
} lazy_job;

static void lazy_task(void* ctx, int64_t t) {
  lazy_job* J = (lazy_job*)ctx;
  const pointset* P = &J->P;
  int64_t i = J->idx[t];
  int32_t rho_i = density_one(P, &J->c, i);
  J->rho_q[t] = rho_i;
  int64_t prev = -1;
  sqd ps;
  ps.si = 0;
  ps.sf = 0.0;
  for (int64_t checks = 0; checks < J->max_checks; ++checks) {
    int64_t next = -1;
    sqd ns;
    ns.si = 0;
    ns.sf = 0.0;
    for (int64_t j = 0; j < P->n; ++j) {
      if (j == i) continue;
      sqd s = sqdist(P, i, j);
      if (prev >= 0 && !sqd_less(P, ps, prev, s, j)) continue; /* not above prev */
      if (next < 0 || sqd_less(P, s, j, ns, next)) {
        next = j;
        ns = s;
      }
    }
    if (next < 0) { /* nobody is higher: i is the highest point */
      J->lam[t] = -1;
      J->delta[t] = INFINITY;
      J->status[t] = 1;
      return;
    }
    int32_t rho_next = density_one(P, &J->c, next);
    if (higher(P, rho_next, next, rho_i, i)) {
      J->lam[t] = (int32_t)next;
      J->delta[t] = sqrt(sqd_value(ns));
      J->status[t] = 1;
      return;
    }
    prev = next;
    ps = ns;
  }
  J->lam[t] = -1;
  J->delta[t] = NAN;
  J->status[t] = 0;
}

int orc_dependent_at(const void* pts, int dtype, int64_t n, int d, double d_cut,
                     const int64_t* idx, int64_t m, int64_t max_checks, int variant,
                     int threads, int32_t* lambda_out, double* delta_out, int32_t* rho_out,
                     int8_t* status_out) {
  if (!pts || n < 0 || d < 1 || !idx || m < 0 || !lambda_out || !delta_out || !rho_out ||
      !status_out)
    return -1;
  lazy_job J;
  J.P.pts = pts;
  J.P.dtype = dtype;
  J.P.n = n;
  J.P.d = d;
  J.P.variant = variant;
  J.c = make_cutoff(d_cut);
  J.idx = idx;
  J.max_checks = max_checks;
  J.lam = lambda_out;
  J.delta = delta_out;
  J.rho_q = rho_out;
  J.status = status_out;
  parallel_for(m, threads, lazy_task, &J);
  return 0;
}

/* ---- exported: labels ----------------------------------------------------
 *
 * Definitions 4-5 and the assignment rule: follow dependent pointers from each
 * point until a center is met; every point on the way takes that center's
 * index.  Returns -2 if a pointer chain from a non-noise, non-center point
 * leaves the point set, reaches a noise point or does not end within n steps.
 */
int orc_cluster(int64_t n, const int32_t* rho, const int32_t* lambda, const double* delta,
                int32_t rho_noise, int32_t rho_min, double delta_min, int variant,
                int32_t* label_out) {
  if (n < 0 || !rho || !lambda || !delta || !label_out) return -1;
  const int check_rho_min = !(variant & ORC_VAR_CENTER_NO_RHO_MIN);
  /* -3 = not yet known */
  for (int64_t i = 0; i < n; ++i) {
    if (rho[i] < rho_noise)
      label_out[i] = -1;                                  /* Definition 4 */
    else if (lambda[i] < 0 ||
             ((!check_rho_min || rho[i] >= rho_min) && delta[i] >= delta_min))
      label_out[i] = (int32_t)i;                          /* Definition 5 */
    else
      label_out[i] = -3;
  }
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (label_out[i] != -3) continue;
    /* walk to the first point whose label is known */
    int64_t cur = i;
    int64_t steps = 0;
    while (label_out[cur] == -3) {
      int64_t nxt = lambda[cur];
      if (nxt < 0 || nxt >= n || ++steps > n) {
        rc = -2;
        break;
      }
      cur = nxt;
    }
    int32_t lab = (rc == 0) ? label_out[cur] : -1;
    if (rc == 0 && lab == -1) rc = -2; /* a non-noise chain ended at noise */
    /* second walk: write the label along the path */
    cur = i;
    steps = 0;
    while (label_out[cur] == -3 && steps++ <= n) {
      label_out[cur] = lab;
      int64_t nxt = lambda[cur];
      if (nxt < 0 || nxt >= n) break;
      cur = nxt;
    }
    if (rc) return rc;
  }
  return rc;
}

/* ---- exported: k-th nearest squared distance (parameter selection) --------
 *
 * For the chosen points, the k-th smallest squared distance to any point of
 * the set, the point itself counted first (k = 1 gives 0).  Used only to pick
 * workload parameters such as a d_cut with a given median density.
 */
typedef struct {
  pointset P;
  const int64_t* idx;
  int k;
  double* out;
} knn_job;

static void knn_task(void* ctx, int64_t t) {
  knn_job* J = (knn_job*)ctx;
  const pointset* P = &J->P;
  int64_t i = J->idx[t];
  int k = J->k;
  double* best = (double*)malloc(sizeof(double) * (size_t)k); /* ascending */
  int have = 0;
  for (int64_t j = 0; j < P->n; ++j) {
    double s = sqd_value(sqdist(P, i, j));
    if (have == k && s >= best[k - 1]) continue;
    int pos = have < k ? have++ : k - 1;
    while (pos > 0 && best[pos - 1] > s) {
      best[pos] = best[pos - 1];
      --pos;
    }
    best[pos] = s;
  }
  J->out[t] = have == k ? best[k - 1] : INFINITY;
  free(best);
}

int orc_kth_sqdist(const void* pts, int dtype, int64_t n, int d, const int64_t* idx, int64_t m,
                   int k, int threads, double* out) {
  if (!pts || n < 0 || d < 1 || !idx || m < 0 || k < 1 || !out) return -1;
  knn_job J;
  J.P.pts = pts;
  J.P.dtype = dtype;
  J.P.n = n;
  J.P.d = d;
  J.P.variant = 0;
  J.idx = idx;
  J.k = k;
  J.out = out;
  parallel_for(m, threads, knn_task, &J);
  return 0;
}

int orc_threads(int threads) { return resolve_threads(threads); }
