/*
 * Seeded synthetic graph generators shared by the CPU oracle, the tests and
 * the benchmark.  This module holds no arithmetic of the clique method: it only
 * draws random graphs and turns edge lists into simple symmetric CSR.
 *
 * Every random number is a pure function of (seed, stream, counter): the
 * SplitMix64 finaliser (Steele, Lea, Flood 2014) applied to a Weyl sequence.
 * Floating point uses only IEEE +, -, *, / and comparisons, in a fixed order,
 * and must be compiled with -ffp-contract=off, so x86-64 and AArch64 builds
 * produce bit-identical graphs.  The logarithm and exponential are the
 * textbook series below (atanh series for log, Taylor series for exp), not the
 * C library's, for the same reason.
 *
 * Families (the workload shapes of the paper's social/information networks):
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004), no noise, random relabelling;
 *   - Chung-Lu with i.i.d. Pareto expected degrees, ball-dropping sampling;
 *   - Erdos-Renyi G(n, p) by geometric skipping (Batagelj, Brandes 2005);
 *   - a planted clique of k distinct uniform vertices on top of any of them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---------------------------------------------------------------- RNG --- */

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + 0x632BE59BD9B4E019ULL) ^ (stream * 0x9E3779B97F4A7C15ULL + 0x2545F4914F6CDD1DULL));
}

uint64_t gg_rand(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

/* uniform double in [0, 1) with 53 random bits (exact conversion) */
static inline double u01(uint64_t key, uint64_t ctr) {
  return (double)(gg_rand(key, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, n), multiply-shift on 32-bit halves (exact) */
static inline uint64_t below(uint64_t r, uint64_t n) {
  if (n <= 0xFFFFFFFFULL) return ((r >> 32) * n) >> 32;
  return r % n;
}

/* ------------------------------------------- deterministic log and exp --- */

static const double LN2 = 0.69314718055994530942;

/* natural log for x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(s), s = (m - 1)/(m + 1), |s| < 0.1716 */
double gg_log(double x) {
  int e = 0;
  double m = x;
  while (m >= 1.4142135623730951) { m *= 0.5; e++; }
  while (m < 0.70710678118654752) { m *= 2.0; e--; }
  double s = (m - 1.0) / (m + 1.0);
  double s2 = s * s, term = s, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= s2; }
  return 2.0 * sum + (double)e * LN2;
}

/* exp x = 2^k e^r, r = x - k ln 2, |r| <= ln2/2, Taylor series to r^24 */
double gg_exp(double x) {
  double kd = x / LN2;
  long k = (long)(kd < 0 ? kd - 0.5 : kd + 0.5);
  double r = x - (double)k * LN2;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 24; i++) { term = term * r / (double)i; sum += term; }
  while (k > 0) { sum *= 2.0; k--; }
  while (k < 0) { sum *= 0.5; k++; }
  return sum;
}

/* ------------------------------------------------------ thread helper --- */

typedef struct {
  void (*fn)(void *, int64_t, int64_t);
  void *arg;
  int64_t lo, hi;
} gg_task;

static void *gg_run(void *p) {
  gg_task *t = (gg_task *)p;
  t->fn(t->arg, t->lo, t->hi);
  return NULL;
}

static void par_for(int threads, int64_t n, void (*fn)(void *, int64_t, int64_t), void *arg) {
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  if (threads == 1 || n < 4096) { fn(arg, 0, n); return; }
  pthread_t th[64];
  gg_task tk[64];
  for (int i = 0; i < threads; i++) {
    tk[i].fn = fn; tk[i].arg = arg;
    tk[i].lo = n * i / threads; tk[i].hi = n * (i + 1) / threads;
    pthread_create(&th[i], NULL, gg_run, &tk[i]);
  }
  for (int i = 0; i < threads; i++) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------- R-MAT --- */

typedef struct {
  int scale; uint64_t key; uint32_t ta, tab, tabc;
  const int32_t *perm; int32_t *src, *dst;
} rmat_arg;

static void rmat_body(void *p, int64_t lo, int64_t hi) {
  rmat_arg *a = (rmat_arg *)p;
  for (int64_t e = lo; e < hi; e++) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < a->scale; l++) {
      uint32_t x;
      if ((l & 1) == 0) { r = gg_rand(a->key, (uint64_t)e * 32 + (uint64_t)(l >> 1)); x = (uint32_t)r; }
      else x = (uint32_t)(r >> 32);
      u <<= 1; v <<= 1;
      if (x < a->ta) { }
      else if (x < a->tab) { v |= 1; }
      else if (x < a->tabc) { u |= 1; }
      else { u |= 1; v |= 1; }
    }
    a->src[e] = a->perm[u];
    a->dst[e] = a->perm[v];
  }
}

/* uniform random permutation of [0, n) (Fisher-Yates) */
void gg_permutation(int64_t n, uint64_t key, int32_t *perm) {
  for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)below(gg_rand(key, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

/* nedges sampled R-MAT edges over 2^scale vertices.  Quadrant choice per level
 * compares a 32-bit uniform against round(p * 2^32) thresholds. */
int gg_rmat_edges(int scale, int64_t nedges, double a, double b, double c, uint64_t seed,
                  int threads, int32_t *src, int32_t *dst) {
  if (scale < 1 || scale > 30) return -1;
  int64_t n = (int64_t)1 << scale;
  int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!perm) return -3;
  gg_permutation(n, gg_key(seed, 11), perm);
  rmat_arg arg;
  arg.scale = scale; arg.key = gg_key(seed, 12);
  arg.ta = (uint32_t)(a * 4294967296.0 + 0.5);
  arg.tab = (uint32_t)((a + b) * 4294967296.0 + 0.5);
  arg.tabc = (uint32_t)((a + b + c) * 4294967296.0 + 0.5);
  arg.perm = perm; arg.src = src; arg.dst = dst;
  par_for(threads, nedges, rmat_body, &arg);
  free(perm);
  return 0;
}

/* ---------------------------------------------------------- Chung-Lu --- */

/* Pareto expected degrees: w = xmin * exp(E / (gamma - 1)), E ~ Exp(1),
 * capped at cap, xmin found by bisection so that mean(w) == mean. */
int gg_chung_lu_weights(int64_t n, double gamma, double mean, double cap, uint64_t seed, double *w) {
  if (n < 1 || gamma <= 1.0 || mean <= 0.0) return -1;
  uint64_t key = gg_key(seed, 21);
  double inv = 1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; i++) {
    double U = u01(key, (uint64_t)i);
    w[i] = gg_exp(-gg_log(1.0 - U) * inv); /* >= 1 */
  }
  double lo = 0.0, hi = mean;
  for (int it = 0; it < 100; it++) {
    double mid = 0.5 * (lo + hi), s = 0.0;
    for (int64_t i = 0; i < n; i++) { double x = mid * w[i]; s += (cap > 0 && x > cap) ? cap : x; }
    if (s / (double)n < mean) lo = mid; else hi = mid;
  }
  double xmin = 0.5 * (lo + hi);
  for (int64_t i = 0; i < n; i++) { double x = xmin * w[i]; w[i] = (cap > 0 && x > cap) ? cap : x; }
  return 0;
}

typedef struct {
  int64_t n; uint64_t key; const double *prob; const int32_t *alias; int32_t *src, *dst;
} cl_arg;

static void cl_body(void *p, int64_t lo, int64_t hi) {
  cl_arg *a = (cl_arg *)p;
  for (int64_t e = lo; e < hi; e++) {
    for (int s = 0; s < 2; s++) {
      uint64_t ctr = ((uint64_t)e * 2 + (uint64_t)s) * 2;
      int64_t i = (int64_t)below(gg_rand(a->key, ctr), (uint64_t)a->n);
      double U = u01(a->key, ctr + 1);
      int32_t v = (U < a->prob[i]) ? (int32_t)i : a->alias[i];
      if (s == 0) a->src[e] = v; else a->dst[e] = v;
    }
  }
}

/* Vose alias table for weights w, then nedges endpoint pairs each drawn
 * with probability proportional to w (ball dropping). */
int gg_chung_lu_edges(int64_t n, const double *w, int64_t nedges, uint64_t seed, int threads,
                      int32_t *src, int32_t *dst) {
  double *prob = (double *)malloc((size_t)n * sizeof(double));
  int32_t *alias = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *small = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *large = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!prob || !alias || !small || !large) { free(prob); free(alias); free(small); free(large); return -3; }
  double tot = 0.0;
  for (int64_t i = 0; i < n; i++) tot += w[i];
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; i++) {
    prob[i] = w[i] * (double)n / tot;
    alias[i] = (int32_t)i;
    if (prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = small[--ns], l = large[nl - 1];
    alias[s] = l;
    prob[l] = (prob[l] + prob[s]) - 1.0;
    if (prob[l] < 1.0) { nl--; small[ns++] = l; }
  }
  while (nl > 0) prob[large[--nl]] = 1.0;
  while (ns > 0) prob[small[--ns]] = 1.0;
  cl_arg arg = {n, gg_key(seed, 22), prob, alias, src, dst};
  par_for(threads, nedges, cl_body, &arg);
  free(prob); free(alias); free(small); free(large);
  return 0;
}

/* ------------------------------------------------------ Erdos-Renyi --- */

/* G(n, p) by geometric skipping over the pairs (v, w), w < v.  Writes at most
 * cap edges; returns the number of edges, or -4 if cap was too small. */
int64_t gg_er_edges(int64_t n, double p, uint64_t seed, int32_t *src, int32_t *dst, int64_t cap) {
  if (n < 1) return 0;
  int64_t m = 0;
  if (p >= 1.0) {
    for (int64_t v = 1; v < n; v++)
      for (int64_t w = 0; w < v; w++) {
        if (m >= cap) return -4;
        src[m] = (int32_t)v; dst[m] = (int32_t)w; m++;
      }
    return m;
  }
  if (p <= 0.0) return 0;
  uint64_t key = gg_key(seed, 31);
  double lq = gg_log(1.0 - p);
  int64_t v = 1, w = -1;
  uint64_t ctr = 0;
  while (v < n) {
    double U = u01(key, ctr++);
    double skip = gg_log(1.0 - U) / lq;
    w = w + 1 + (int64_t)skip;
    while (w >= v && v < n) { w -= v; v++; }
    if (v < n) {
      if (m >= cap) return -4;
      src[m] = (int32_t)v; dst[m] = (int32_t)w; m++;
    }
  }
  return m;
}

/* ------------------------------------------------------ planted clique --- */

/* k distinct uniform vertices of [0, n) (rejection on a bitmap); writes the
 * sorted members to members[] and the k(k-1)/2 pairs to src/dst. */
int gg_planted(int64_t n, int64_t k, uint64_t seed, int32_t *members, int32_t *src, int32_t *dst) {
  if (k > n || k < 0) return -1;
  uint8_t *used = (uint8_t *)calloc((size_t)n, 1);
  if (!used) return -3;
  uint64_t key = gg_key(seed, 41), ctr = 0;
  for (int64_t i = 0; i < k;) {
    int64_t v = (int64_t)below(gg_rand(key, ctr++), (uint64_t)n);
    if (!used[v]) { used[v] = 1; i++; }
  }
  int64_t j = 0;
  for (int64_t v = 0; v < n; v++) if (used[v]) members[j++] = (int32_t)v;
  free(used);
  int64_t e = 0;
  for (int64_t a = 0; a < k; a++)
    for (int64_t b = a + 1; b < k; b++) { src[e] = members[a]; dst[e] = members[b]; e++; }
  return 0;
}

/* ---------------------------------------------------- edges -> CSR --- */

static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

typedef struct { int64_t *rp; int32_t *col; int64_t *newdeg; } sort_arg;

static void sort_body(void *p, int64_t lo, int64_t hi) {
  sort_arg *a = (sort_arg *)p;
  for (int64_t v = lo; v < hi; v++) {
    int32_t *r = a->col + a->rp[v];
    int64_t d = a->rp[v + 1] - a->rp[v];
    if (d > 1) qsort(r, (size_t)d, sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t i = 0; i < d; i++) if (i == 0 || r[i] != r[i - 1]) r[k++] = r[i];
    a->newdeg[v] = k;
  }
}

/* Symmetrise, drop self-loops and duplicates, sort rows ascending.
 * row_ptr has n+1 entries; col must hold 2*m entries (the result uses the
 * first row_ptr[n] of them).  Returns row_ptr[n] (the CSR entry count). */
/* Endpoint counts and the scatter into rows run in parallel with atomic
 * counters: the order of entries inside a row then depends on timing, but
 * every row is sorted and deduplicated afterwards, so the CSR does not. */
typedef struct { int64_t n; const int32_t *src, *dst; int64_t *cnt; int32_t *col; } edge_arg;

static void count_body(void *p, int64_t lo, int64_t hi) {
  edge_arg *a = (edge_arg *)p;
  for (int64_t e = lo; e < hi; e++) {
    int32_t u = a->src[e], v = a->dst[e];
    if (u == v || u < 0 || v < 0 || u >= a->n || v >= a->n) continue;
    __atomic_fetch_add(&a->cnt[u], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&a->cnt[v], 1, __ATOMIC_RELAXED);
  }
}

static void scatter_body(void *p, int64_t lo, int64_t hi) {
  edge_arg *a = (edge_arg *)p;
  for (int64_t e = lo; e < hi; e++) {
    int32_t u = a->src[e], v = a->dst[e];
    if (u == v || u < 0 || v < 0 || u >= a->n || v >= a->n) continue;
    a->col[__atomic_fetch_add(&a->cnt[u], 1, __ATOMIC_RELAXED)] = v;
    a->col[__atomic_fetch_add(&a->cnt[v], 1, __ATOMIC_RELAXED)] = u;
  }
}

int64_t gg_csr_from_edges(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int threads,
                          int64_t *row_ptr, int32_t *col) {
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -3;
  edge_arg ea = {n, src, dst, cnt, col};
  par_for(threads, m, count_body, &ea);
  int64_t *rp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!rp) { free(cnt); return -3; }
  rp[0] = 0;
  for (int64_t v = 0; v < n; v++) rp[v + 1] = rp[v] + cnt[v];
  for (int64_t v = 0; v < n; v++) cnt[v] = rp[v];
  par_for(threads, m, scatter_body, &ea);
  sort_arg sa = {rp, col, cnt};
  par_for(threads, n, sort_body, &sa);
  /* compact rows in place (rows only move left) */
  row_ptr[0] = 0;
  for (int64_t v = 0; v < n; v++) {
    int64_t d = cnt[v], from = rp[v], to = row_ptr[v];
    if (to != from) memmove(col + to, col + from, (size_t)d * sizeof(int32_t));
    row_ptr[v + 1] = to + d;
  }
  free(cnt); free(rp);
  return row_ptr[n];
}
