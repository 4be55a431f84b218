/*
 * CPU oracle for exact maximum clique (Rossi, Gleich, Gebremedhin, Patwary,
 * "Parallel Maximum Clique Algorithms with Applications to Network Analysis
 * and Storage").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow C that follows the paper's
 * definitions and algorithms step by step (single-threaded, except for the
 * threaded search at the end, which exists to reach the largest inputs).  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg use it; the product path never
 * calls it, and it shares no code, header or table with the CUDA library.
 *
 * Contents and the passage each function follows:
 *   orc_core_numbers      Section 3 (core number K(v), degeneracy), computed by
 *                         the Batagelj-Zaversnik bucket algorithm the paper cites.
 *   orc_greedy_colors     Section 3 (greedy colouring in degeneracy order, L(G)).
 *   orc_heuristic_clique  Algorithm 1 (HeuristicClique), Section 4.1.
 *   orc_max_clique        Algorithm 2 (MaxClique, InitialBranch, Branch),
 *                         Sections 4.2-4.3.
 *   orc_is_clique         the definition of a clique.
 *   orc_max_clique_threads the same exact search by several workers sharing
 *                         the incumbent (Section 4.5), roots in a static
 *                         degeneracy order.
 *   orc_max_clique_part   the same, restricted to one part of a partition of
 *                         the roots (every part_count-th position of a given
 *                         degeneracy order): the search of one rank of several
 *                         that split the roots (Section 4.5 distributes them
 *                         over processors).
 *
 * Readings of points the paper leaves open (each is exact: omega and K do not
 * depend on them):
 *   - Algorithm 1 starts C from {v} (every u in S is a neighbour of v).
 *   - Ties in "decreasing core number" order break by larger degree, then
 *     smaller vertex id.
 *   - InitialBranch returns when K(P) + 1 <= |H| (the tight form of the test;
 *     a clique larger than |H| in N_R(u) needs a |H|-core there).
 *   - Degeneracy order for the InitialBranch colouring: decreasing K_N, ties
 *     by smaller id.  "Natural order" in Branch: increasing vertex id.
 *   - Branch selects the vertex of largest colour (ties: the last in natural
 *     order) and also stops once |C| + colour(u) <= |H| (Tomita's colour
 *     bound), which prunes only branches that cannot beat |H|.
 *   - The main loop's "smallest reduced degree" breaks ties by smaller id; the
 *     wall-clock periodic rebuild is left out (it changes work only).
 *   - n = 0 gives omega = 0; a graph without edges gives omega = 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_BUFFER (-4)

/* ------------------------------------------------------------ helpers --- */

static int adjacent(const int64_t *rp, const int32_t *ci, int32_t a, int32_t b) {
  /* binary search b in the sorted row of a (choose the shorter row) */
  int64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
  if (db < da) { int32_t t = a; a = b; b = t; }
  int64_t lo = rp[a], hi = rp[a + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (ci[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo < rp[a + 1] && ci[lo] == b;
}

int orc_is_clique(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *vs, int32_t k) {
  for (int32_t i = 0; i < k; i++) {
    if (vs[i] < 0 || vs[i] >= n) return 0;
    for (int32_t j = i + 1; j < k; j++) {
      if (vs[i] == vs[j]) return 0;
      if (!adjacent(rp, ci, vs[i], vs[j])) return 0;
    }
  }
  return 1;
}

/* ----------------------------------------------------- core numbers --- */

/* Batagelj-Zaversnik: visit vertices in nondecreasing current degree (bucket
 * sort), and for each visited v lower the degree of every neighbour whose
 * degree is still larger.  The final degree of v is its core number K(v).
 * If order_out is not NULL it receives the visiting (degeneracy) order. */
int orc_core_numbers(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *core, int32_t *order_out) {
  if (n < 0) return ORC_ERR_ARG;
  if (n == 0) return ORC_OK;
  int64_t md = 0;
  int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int32_t *vert = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!deg || !pos || !vert) { free(deg); free(pos); free(vert); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; v++) { deg[v] = rp[v + 1] - rp[v]; if (deg[v] > md) md = deg[v]; }
  int64_t *bin = (int64_t *)calloc((size_t)md + 1, sizeof(int64_t));
  if (!bin) { free(deg); free(pos); free(vert); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; v++) bin[deg[v]]++;
  int64_t start = 0;
  for (int64_t d = 0; d <= md; d++) { int64_t num = bin[d]; bin[d] = start; start += num; }
  for (int64_t v = 0; v < n; v++) { pos[v] = bin[deg[v]]; vert[pos[v]] = (int32_t)v; bin[deg[v]]++; }
  for (int64_t d = md; d >= 1; d--) bin[d] = bin[d - 1];
  bin[0] = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = vert[i];
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
      int32_t u = ci[e];
      if (deg[u] > deg[v]) {
        int64_t du = deg[u], pu = pos[u], pw = bin[du];
        int32_t w = vert[pw];
        if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
        bin[du]++;
        deg[u]--;
      }
    }
  }
  for (int64_t v = 0; v < n; v++) core[v] = (int32_t)deg[v];
  if (order_out) memcpy(order_out, vert, (size_t)n * sizeof(int32_t));
  free(deg); free(pos); free(vert); free(bin);
  return ORC_OK;
}

/* --------------------------------------------------- greedy colouring --- */

/* Greedy colouring in the given vertex order: each vertex takes the smallest
 * colour (1, 2, ...) that no already-coloured neighbour has.  Returns the
 * number of colours L; colors_out (nullable) receives each vertex's colour. */
int32_t orc_greedy_colors(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *order, int32_t *colors_out) {
  if (n <= 0) return 0;
  int32_t *col = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  int64_t *mark = (int64_t *)malloc(((size_t)n + 2) * sizeof(int64_t));
  if (!col || !mark) { free(col); free(mark); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < n + 2; i++) mark[i] = -1;
  int32_t L = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = order[i];
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
      int32_t c = col[ci[e]];
      if (c > 0 && c <= n + 1) mark[c] = i;
    }
    int32_t c = 1;
    while (mark[c] == i) c++;
    col[v] = c;
    if (c > L) L = c;
  }
  if (colors_out) memcpy(colors_out, col, (size_t)n * sizeof(int32_t));
  free(col); free(mark);
  return L;
}

/* ---------------------------------------------- heuristic (Algorithm 1) --- */

typedef struct { int32_t v; int32_t k; int64_t d; } vkey;

/* decreasing core number, then decreasing degree, then increasing id */
static int cmp_vkey(const void *x, const void *y) {
  const vkey *a = (const vkey *)x, *b = (const vkey *)y;
  if (a->k != b->k) return a->k > b->k ? -1 : 1;
  if (a->d != b->d) return a->d > b->d ? -1 : 1;
  return (a->v > b->v) - (a->v < b->v);
}

/* Algorithm 1.  mode 0: the algorithm as printed (running max, candidates S
 * filtered by K >= max, vertices with K(v) < max skipped).  mode 1: the same
 * greedy grown from every vertex with max held at 0 (S = all neighbours); the
 * result is the largest such clique, ties to the smallest start vertex.
 * Writes the clique (sorted ascending) to H (capacity cap) and its size. */
int orc_heuristic_clique(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *core, int mode,
                         int32_t *H, int32_t cap, int32_t *size_out) {
  if (n < 0 || (mode != 0 && mode != 1)) return ORC_ERR_ARG;
  *size_out = 0;
  if (n == 0) return ORC_OK;
  vkey *ord = (vkey *)malloc((size_t)n * sizeof(vkey));
  int64_t maxd = 0;
  for (int64_t v = 0; v < n; v++) if (rp[v + 1] - rp[v] > maxd) maxd = rp[v + 1] - rp[v];
  vkey *S = (vkey *)malloc(((size_t)maxd + 1) * sizeof(vkey));
  int32_t *C = (int32_t *)malloc(((size_t)maxd + 2) * sizeof(int32_t));
  int32_t *best = (int32_t *)malloc(((size_t)maxd + 2) * sizeof(int32_t));
  if (!ord || !S || !C || !best) { free(ord); free(S); free(C); free(best); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; v++) { ord[v].v = (int32_t)v; ord[v].k = core[v]; ord[v].d = rp[v + 1] - rp[v]; }
  qsort(ord, (size_t)n, sizeof(vkey), cmp_vkey);
  int32_t max = 0, best_v = -1;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = ord[i].v;
    int32_t T = (mode == 0) ? max : 0;
    if (mode == 0 && core[v] < max) continue;
    if (mode == 1 && core[v] + 1 < max) continue; /* |C| <= K(v) + 1 cannot reach max */
    int64_t ns = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
      int32_t u = ci[e];
      if (core[u] >= T) { S[ns].v = u; S[ns].k = core[u]; S[ns].d = rp[u + 1] - rp[u]; ns++; }
    }
    qsort(S, (size_t)ns, sizeof(vkey), cmp_vkey);
    int32_t c = 0;
    C[c++] = v;
    for (int64_t j = 0; j < ns; j++) {
      int32_t u = S[j].v, ok = 1;
      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(rp, ci, u, C[t]);
      if (ok) C[c++] = u;
    }
    if (c > max || (mode == 1 && c == max && v < best_v)) {
      max = c; best_v = v;
      memcpy(best, C, (size_t)c * sizeof(int32_t));
    }
  }
  *size_out = max;
  int rc = ORC_OK;
  if (max > cap) rc = ORC_ERR_BUFFER;
  else {
    /* sort ascending */
    for (int32_t a = 1; a < max; a++) {
      int32_t x = best[a], b = a - 1;
      while (b >= 0 && best[b] > x) { best[b + 1] = best[b]; b--; }
      best[b + 1] = x;
    }
    memcpy(H, best, (size_t)max * sizeof(int32_t));
  }
  free(ord); free(S); free(C); free(best);
  return rc;
}

/* -------------------------------------------- exact search (Algorithm 2) --- */

typedef struct {
  /* explicitly pruned graph (vertices with K >= |H| after the heuristic) */
  int64_t n;
  const int64_t *rp;
  const int32_t *ci;
  const int32_t *K;     /* core numbers in the pruned graph's numbering */
  const int32_t *orig;  /* original vertex id */
  uint8_t *searched;    /* X: vertices whose InitialBranch has finished */
  /* incumbent H */
  int32_t *H;           /* original ids */
  int32_t hsize;
  /* InitialBranch workspace: P's induced subgraph as a byte matrix */
  int32_t *P;           /* pruned-graph ids of P */
  int32_t np;
  uint8_t *adj;         /* np x np */
  int32_t *C;           /* current clique (indices into P) */
  int64_t nodes;        /* Branch calls */
  int64_t ib_calls, ib_full;
  int err;
} mc_state;

static int alive(const mc_state *s, int32_t v) {
  return !s->searched[v] && s->K[v] >= s->hsize;
}

/* greedy colouring of the vertices idx[0..cnt) (indices into P) in that order;
 * writes colours, returns the number of colours */
static int32_t color_list(const mc_state *s, const int32_t *idx, int32_t cnt, int32_t *colors, int32_t *scratch) {
  int32_t L = 0;
  for (int32_t i = 0; i < cnt; i++) {
    int32_t a = idx[i];
    for (int32_t c = 0; c <= cnt + 1; c++) scratch[c] = 0;
    for (int32_t j = 0; j < i; j++)
      if (s->adj[(int64_t)a * s->np + idx[j]]) scratch[colors[j]] = 1;
    int32_t c = 1;
    while (scratch[c]) c++;
    colors[i] = c;
    if (c > L) L = c;
  }
  return L;
}

/* Branch(C, P): P = idx[0..cnt) in natural order with their colours. */
static void branch(mc_state *s, int32_t csize, int32_t *idx, int32_t *colors, int32_t cnt) {
  s->nodes++;
  int32_t *pidx = (int32_t *)malloc(((size_t)cnt + 1) * sizeof(int32_t));
  int32_t *pcol = (int32_t *)malloc(((size_t)cnt + 1) * sizeof(int32_t));
  int32_t *scr = (int32_t *)malloc(((size_t)cnt + 3) * sizeof(int32_t));
  if (!pidx || !pcol || !scr) { s->err = ORC_ERR_OOM; free(pidx); free(pcol); free(scr); return; }
  while (cnt > 0 && cnt + csize > s->hsize) {
    /* select the vertex of largest colour (last one on ties) and remove it */
    int32_t at = 0;
    for (int32_t i = 1; i < cnt; i++) if (colors[i] >= colors[at]) at = i;
    int32_t u = idx[at], cu = colors[at];
    for (int32_t i = at; i + 1 < cnt; i++) { idx[i] = idx[i + 1]; colors[i] = colors[i + 1]; }
    cnt--;
    if (csize + cu <= s->hsize) break;
    s->C[csize] = u;
    int32_t c2 = csize + 1;
    /* P' = P intersected with N_R(u) (alive neighbours of u) */
    int32_t np2 = 0;
    for (int32_t i = 0; i < cnt; i++) {
      int32_t w = idx[i];
      if (s->adj[(int64_t)u * s->np + w] && alive(s, s->P[w])) pidx[np2++] = w;
    }
    if (np2 > 0) {
      int32_t L = color_list(s, pidx, np2, pcol, scr);
      if (c2 + L > s->hsize) {
        branch(s, c2, pidx, pcol, np2);
        if (s->err) break;
      }
    } else if (c2 > s->hsize) {
      /* C' is maximal and larger than H: new incumbent.  Vertices with
       * K < |H| become implicitly removed through alive(). */
      for (int32_t i = 0; i < c2; i++) s->H[i] = s->orig[s->P[s->C[i]]];
      s->hsize = c2;
    }
  }
  free(pidx); free(pcol); free(scr);
}

/* core numbers of the np-vertex graph given by the byte matrix (BZ again,
 * on the small graph) */
static void small_cores(const uint8_t *adj, int32_t np, const uint8_t *in, int32_t *kn) {
  /* simple peeling: repeatedly remove a vertex of minimum remaining degree */
  int32_t *deg = (int32_t *)malloc((size_t)np * sizeof(int32_t));
  uint8_t *gone = (uint8_t *)malloc((size_t)np);
  for (int32_t a = 0; a < np; a++) {
    gone[a] = !in[a];
    deg[a] = 0;
  }
  for (int32_t a = 0; a < np; a++)
    if (in[a])
      for (int32_t b = 0; b < np; b++) if (in[b] && adj[(int64_t)a * np + b]) deg[a]++;
  int32_t k = 0;
  for (;;) {
    int32_t at = -1;
    for (int32_t a = 0; a < np; a++) if (!gone[a] && (at < 0 || deg[a] < deg[at])) at = a;
    if (at < 0) break;
    if (deg[at] > k) k = deg[at];
    kn[at] = k;
    gone[at] = 1;
    for (int32_t b = 0; b < np; b++) if (!gone[b] && adj[(int64_t)at * np + b]) deg[b]--;
  }
  free(deg); free(gone);
}

typedef struct { int32_t i; int32_t kn; int32_t id; } knkey;
static int cmp_knkey(const void *x, const void *y) {
  const knkey *a = (const knkey *)x, *b = (const knkey *)y;
  if (a->kn != b->kn) return a->kn > b->kn ? -1 : 1;
  return (a->id > b->id) - (a->id < b->id);
}

/* InitialBranch(u) */
static void initial_branch(mc_state *s, int32_t u) {
  s->ib_calls++;
  /* P = N_R(u): u and its alive neighbours, in increasing id */
  int32_t np = 0;
  int inserted = 0;
  for (int64_t e = s->rp[u]; e < s->rp[u + 1]; e++) {
    int32_t w = s->ci[e];
    if (!inserted && w > u) { s->P[np++] = u; inserted = 1; }
    if (alive(s, w)) s->P[np++] = w;
  }
  if (!inserted) s->P[np++] = u;
  if (np <= s->hsize) return;
  s->ib_full++;
  s->np = np;
  s->adj = (uint8_t *)calloc((size_t)np * (size_t)np, 1);
  int32_t *kn = (int32_t *)malloc((size_t)np * sizeof(int32_t));
  uint8_t *in = (uint8_t *)malloc((size_t)np);
  int32_t *idx = (int32_t *)malloc((size_t)np * sizeof(int32_t));
  int32_t *col = (int32_t *)malloc((size_t)np * sizeof(int32_t));
  int32_t *scr = (int32_t *)malloc(((size_t)np + 3) * sizeof(int32_t));
  knkey *ord = (knkey *)malloc((size_t)np * sizeof(knkey));
  if (!s->adj || !kn || !in || !idx || !col || !scr || !ord) {
    s->err = ORC_ERR_OOM;
    goto done;
  }
  /* induced subgraph of P: binary search of P's members in each row */
  for (int32_t a = 0; a < np; a++)
    for (int32_t b = a + 1; b < np; b++)
      if (adjacent(s->rp, s->ci, s->P[a], s->P[b])) {
        s->adj[(int64_t)a * np + b] = 1;
        s->adj[(int64_t)b * np + a] = 1;
      }
  for (int32_t a = 0; a < np; a++) in[a] = 1;
  small_cores(s->adj, np, in, kn);
  int32_t KP = 0;
  for (int32_t a = 0; a < np; a++) if (kn[a] > KP) KP = kn[a];
  if (KP + 1 <= s->hsize) goto done;
  /* remove vertices with K_N < |H| */
  int32_t cnt = 0;
  for (int32_t a = 0; a < np; a++)
    if (kn[a] >= s->hsize) { ord[cnt].i = a; ord[cnt].kn = kn[a]; ord[cnt].id = s->P[a]; cnt++; }
  /* colour in degeneracy order (decreasing K_N) */
  qsort(ord, (size_t)cnt, sizeof(knkey), cmp_knkey);
  for (int32_t j = 0; j < cnt; j++) idx[j] = ord[j].i;
  int32_t L = color_list(s, idx, cnt, col, scr);
  if (L <= s->hsize) goto done;
  /* Branch({}, P) with P in natural order carrying those colours */
  {
    int32_t *nat = (int32_t *)malloc((size_t)cnt * sizeof(int32_t));
    int32_t *ncol = (int32_t *)malloc((size_t)cnt * sizeof(int32_t));
    int32_t *cof = (int32_t *)malloc((size_t)np * sizeof(int32_t));
    if (!nat || !ncol || !cof) { s->err = ORC_ERR_OOM; free(nat); free(ncol); free(cof); goto done; }
    for (int32_t a = 0; a < np; a++) cof[a] = 0;
    for (int32_t j = 0; j < cnt; j++) cof[idx[j]] = col[j];
    int32_t c = 0;
    for (int32_t a = 0; a < np; a++) if (kn[a] >= s->hsize) { nat[c] = a; ncol[c] = cof[a]; c++; }
    branch(s, 0, nat, ncol, c);
    free(nat); free(ncol); free(cof);
  }
done:
  free(s->adj); s->adj = NULL;
  free(kn); free(in); free(idx); free(col); free(scr); free(ord);
}

typedef struct {
  int64_t pruned_n;       /* vertices left after the explicit core pruning */
  int64_t initial_branch; /* InitialBranch calls */
  int64_t full_branch;    /* InitialBranch calls that passed the |P| <= |H| test */
  int64_t nodes;          /* Branch calls */
  int32_t heuristic;      /* |H| of Algorithm 1 */
  int32_t max_core;       /* K(G) */
} orc_stats;

/* Algorithm 2, MaxClique(G).  omega_out gets omega(G); witness (capacity cap)
 * a maximum clique, sorted ascending. */
int orc_max_clique(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *omega_out, int32_t *witness,
                   int32_t cap, orc_stats *st) {
  if (n < 0) return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  *omega_out = 0;
  if (n == 0) return ORC_OK;
  int rc = ORC_OK;
  int32_t *K0 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!K0) return ORC_ERR_OOM;
  orc_core_numbers(n, rp, ci, K0, NULL);
  int32_t kmax = 0;
  for (int64_t v = 0; v < n; v++) if (K0[v] > kmax) kmax = K0[v];
  st->max_core = kmax;
  int32_t *H = (int32_t *)malloc(((size_t)kmax + 2) * sizeof(int32_t));
  int32_t hs = 0;
  orc_heuristic_clique(n, rp, ci, K0, 0, H, kmax + 2, &hs);
  st->heuristic = hs;
  /* remove (explicitly) vertices with K(v) < |H| */
  int32_t *newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t n2 = 0, nnz2 = 0;
  for (int64_t v = 0; v < n; v++) newid[v] = (K0[v] >= hs) ? (int32_t)n2++ : -1;
  int64_t *rp2 = (int64_t *)malloc(((size_t)n2 + 1) * sizeof(int64_t));
  int32_t *orig = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  int32_t *K2 = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  rp2[0] = 0;
  for (int64_t v = 0; v < n; v++) if (newid[v] >= 0) {
    int64_t d = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) if (newid[ci[e]] >= 0) d++;
    orig[newid[v]] = (int32_t)v; K2[newid[v]] = K0[v];
    rp2[newid[v] + 1] = rp2[newid[v]] + d;
  }
  nnz2 = rp2[n2];
  int32_t *ci2 = (int32_t *)malloc(((size_t)nnz2 + 1) * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++) if (newid[v] >= 0) {
    int64_t o = rp2[newid[v]];
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) if (newid[ci[e]] >= 0) ci2[o++] = newid[ci[e]];
  }
  st->pruned_n = n2;
  mc_state s;
  memset(&s, 0, sizeof(s));
  s.n = n2; s.rp = rp2; s.ci = ci2; s.K = K2; s.orig = orig;
  s.searched = (uint8_t *)calloc((size_t)n2 + 1, 1);
  s.H = (int32_t *)malloc(((size_t)kmax + 2) * sizeof(int32_t));
  memcpy(s.H, H, (size_t)hs * sizeof(int32_t));
  s.hsize = hs;
  int64_t maxd2 = 0;
  for (int64_t v = 0; v < n2; v++) if (rp2[v + 1] - rp2[v] > maxd2) maxd2 = rp2[v + 1] - rp2[v];
  s.P = (int32_t *)malloc(((size_t)maxd2 + 2) * sizeof(int32_t));
  s.C = (int32_t *)malloc(((size_t)maxd2 + 2) * sizeof(int32_t));
  /* reduced degrees in buckets (doubly linked lists) for "smallest reduced degree" */
  int64_t *rd = (int64_t *)malloc(((size_t)n2 + 1) * sizeof(int64_t));
  int32_t *head = (int32_t *)malloc(((size_t)maxd2 + 2) * sizeof(int32_t));
  int32_t *nxt = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  int32_t *prv = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  uint8_t *gone = (uint8_t *)calloc((size_t)n2 + 1, 1);
  /* vertices by increasing core number, for implicit removals when |H| grows */
  int32_t *byk = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  if (!s.searched || !s.H || !s.P || !s.C || !rd || !head || !nxt || !prv || !gone || !byk) { rc = ORC_ERR_OOM; goto out; }
  for (int64_t d = 0; d <= maxd2; d++) head[d] = -1;
  for (int64_t v = n2 - 1; v >= 0; v--) {
    rd[v] = rp2[v + 1] - rp2[v];
    nxt[v] = head[rd[v]]; prv[v] = -1;
    if (head[rd[v]] >= 0) prv[head[rd[v]]] = (int32_t)v;
    head[rd[v]] = (int32_t)v;
  }
  {
    /* counting sort by core */
    int64_t *cnt = (int64_t *)calloc((size_t)kmax + 2, sizeof(int64_t));
    for (int64_t v = 0; v < n2; v++) cnt[K2[v] + 1]++;
    for (int32_t k = 0; k <= kmax; k++) cnt[k + 1] += cnt[k];
    for (int64_t v = 0; v < n2; v++) byk[cnt[K2[v]]++] = (int32_t)v;
    free(cnt);
  }
  int64_t kptr = 0, left = n2, mind = 0;
#define UNLINK(v) do { int32_t _v = (v); \
    if (prv[_v] >= 0) nxt[prv[_v]] = nxt[_v]; else head[rd[_v]] = nxt[_v]; \
    if (nxt[_v] >= 0) prv[nxt[_v]] = prv[_v]; } while (0)
#define LINK(v) do { int32_t _v = (v); prv[_v] = -1; nxt[_v] = head[rd[_v]]; \
    if (head[rd[_v]] >= 0) prv[head[rd[_v]]] = _v; head[rd[_v]] = _v; \
    if (rd[_v] < mind) mind = rd[_v]; } while (0)
#define REMOVE(v) do { int32_t _r = (v); UNLINK(_r); gone[_r] = 1; left--; \
    for (int64_t _e = rp2[_r]; _e < rp2[_r + 1]; _e++) { int32_t _w = ci2[_e]; \
      if (!gone[_w]) { UNLINK(_w); rd[_w]--; LINK(_w); } } } while (0)
  while (left > 0) {
    /* implicit removal of vertices with K(v) < |H| */
    while (kptr < n2 && K2[byk[kptr]] < s.hsize) {
      int32_t v = byk[kptr++];
      if (!gone[v]) { s.searched[v] = 1; REMOVE(v); }
    }
    if (left == 0) break;
    while (head[mind] < 0) mind++;
    /* smallest reduced degree, ties to the smallest id */
    int32_t u = head[mind];
    for (int32_t w = nxt[u]; w >= 0; w = nxt[w]) if (w < u) u = w;
    initial_branch(&s, u);
    if (s.err) { rc = s.err; goto out; }
    s.searched[u] = 1;
    REMOVE(u);
  }
#undef UNLINK
#undef LINK
#undef REMOVE
  st->initial_branch = s.ib_calls;
  st->full_branch = s.ib_full;
  st->nodes = s.nodes;
  *omega_out = s.hsize;
  if (s.hsize > cap) rc = ORC_ERR_BUFFER;
  else {
    for (int32_t a = 1; a < s.hsize; a++) {
      int32_t x = s.H[a], b = a - 1;
      while (b >= 0 && s.H[b] > x) { s.H[b + 1] = s.H[b]; b--; }
      s.H[b + 1] = x;
    }
    memcpy(witness, s.H, (size_t)s.hsize * sizeof(int32_t));
  }
out:
  free(K0); free(H); free(newid); free(rp2); free(orig); free(K2); free(ci2);
  free(s.searched); free(s.H); free(s.P); free(s.C);
  free(rd); free(head); free(nxt); free(prv); free(gone); free(byk);
  return rc;
}

/* ------------------------------ threaded exact search (Section 4.5) --- */

/*
 * orc_max_clique_threads: the exact search of Algorithm 2 run by `threads`
 * workers that share the incumbent, as in the paper's parallel method
 * (Section 4.5: each worker reads the current |H| before every pruning test
 * and raises it under a lock).  It exists for graphs whose single-threaded
 * search above takes hours; it shares no code with the CUDA library either.
 *
 *  1. K(v) and a degeneracy order by Batagelj-Zaversnik (orc_core_numbers);
 *     rank(v) = the position of v in that order.
 *  2. Algorithm 1 as printed, its start vertices handed to the workers in
 *     decreasing core order, with the running maximum shared by all.
 *  3. Vertices with K(v) < |H| removed (Section 4.2); the rest numbered by
 *     rank, each keeping its later neighbours N+(v) (rank(w) > rank(v)).
 *  4. Each worker takes the next root u in rank order and looks for cliques
 *     larger than |H| whose lowest-ranked member is u:
 *       P = {w in N+(u) : K(w) >= |H|}; skip if |P| + 1 <= |H|;
 *       core numbers K_P of the subgraph induced by P -- with u, which is
 *       adjacent to all of P, every one of them is one larger -- so keep
 *       w with K_P(w) + 1 >= |H| and skip if |kept| + 1 <= |H|;
 *       greedy colouring of the kept vertices in decreasing K_P (ties:
 *       smaller vertex id); skip if 1 + L <= |H|;
 *       Branch({u}, kept), with the colour bound, as in orc_max_clique.
 *  Every clique has exactly one lowest-ranked member, so each clique larger
 *  than the final |H| falls in exactly one root's search: omega is exact for
 *  any root order and any interleaving of the workers (only the witness and
 *  the work counts can differ from run to run).
 */
#include <pthread.h>

static int cmp_i32_asc(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

typedef struct {
  /* Algorithm 1 (printed form) over the shared visiting order */
  int64_t n;
  const int64_t *rp;
  const int32_t *ci;
  const int32_t *core;
  const vkey *ord;
  int64_t maxd;
  int64_t next;   /* next position of ord, taken with __atomic_fetch_add */
  int32_t max;    /* running maximum, __atomic loads and stores */
  int32_t *best;  /* its clique, written under mu */
  pthread_mutex_t mu;
  int err;
} th_heur;

static void *heur_worker(void *arg) {
  th_heur *h = (th_heur *)arg;
  vkey *S = (vkey *)malloc(((size_t)h->maxd + 1) * sizeof(vkey));
  int32_t *C = (int32_t *)malloc(((size_t)h->maxd + 2) * sizeof(int32_t));
  if (!S || !C) { h->err = ORC_ERR_OOM; free(S); free(C); return NULL; }
  for (;;) {
    int64_t i = __atomic_fetch_add(&h->next, 1, __ATOMIC_RELAXED);
    if (i >= h->n) break;
    int32_t v = h->ord[i].v;
    int32_t T = __atomic_load_n(&h->max, __ATOMIC_ACQUIRE);
    /* K(v) >= max is the visiting condition; the order is by decreasing
     * core and max only grows, so no later start vertex passes either */
    if (h->core[v] < T) break;
    int64_t ns = 0;
    for (int64_t e = h->rp[v]; e < h->rp[v + 1]; e++) {
      int32_t u = h->ci[e];
      if (h->core[u] >= T) { S[ns].v = u; S[ns].k = h->core[u]; S[ns].d = h->rp[u + 1] - h->rp[u]; ns++; }
    }
    qsort(S, (size_t)ns, sizeof(vkey), cmp_vkey);
    int32_t c = 0;
    C[c++] = v;
    for (int64_t j = 0; j < ns; j++) {
      int32_t u = S[j].v, ok = 1;
      for (int32_t t = 0; t < c && ok; t++) ok = adjacent(h->rp, h->ci, u, C[t]);
      if (ok) C[c++] = u;
    }
    if (c > __atomic_load_n(&h->max, __ATOMIC_ACQUIRE)) {
      pthread_mutex_lock(&h->mu);
      if (c > h->max) {
        memcpy(h->best, C, (size_t)c * sizeof(int32_t));
        __atomic_store_n(&h->max, c, __ATOMIC_RELEASE);
      }
      pthread_mutex_unlock(&h->mu);
    }
  }
  free(S); free(C);
  return NULL;
}

typedef struct {
  int64_t n2;            /* vertices left after the explicit pruning */
  const int64_t *orp;    /* later neighbours (new ids follow rank) */
  const int32_t *oci;
  const int32_t *K;      /* core numbers, new numbering */
  const int32_t *orig;   /* original vertex id */
  int32_t kmax;
  int64_t next;          /* next root, __atomic_fetch_add */
  int32_t best;          /* |H|, __atomic loads and stores */
  int32_t *H;            /* witness in original ids, written under mu */
  pthread_mutex_t mu;
  int64_t ib_calls, ib_full, nodes; /* summed under mu when a worker ends */
  const int32_t *opos;   /* position of each kept vertex in the full order */
  int32_t part_rank, part_count;
  int err;
} th_search;

typedef struct {
  th_search *sh;
  int32_t *mark;   /* per new id: 0, or 1 + its index in P */
  int32_t *P;      /* new ids of P */
  int32_t np;
  uint8_t *adj;    /* np x np byte matrix of G[P] */
  int32_t *C;      /* the current clique, new ids */
  int64_t nodes, ib_calls, ib_full;
  int err;
} th_worker;

static int32_t th_best(const th_worker *w) { return __atomic_load_n(&w->sh->best, __ATOMIC_ACQUIRE); }

/* greedy colouring of idx[0..cnt) (indices into P) in that order */
static int32_t th_color_list(const th_worker *w, const int32_t *idx, int32_t cnt, int32_t *colors, int32_t *scratch) {
  int32_t L = 0;
  for (int32_t i = 0; i < cnt; i++) {
    int32_t a = idx[i];
    for (int32_t c = 0; c <= cnt + 1; c++) scratch[c] = 0;
    for (int32_t j = 0; j < i; j++)
      if (w->adj[(int64_t)a * w->np + idx[j]]) scratch[colors[j]] = 1;
    int32_t c = 1;
    while (scratch[c]) c++;
    colors[i] = c;
    if (c > L) L = c;
  }
  return L;
}

static void th_raise(th_worker *w, int32_t size) {
  th_search *sh = w->sh;
  pthread_mutex_lock(&sh->mu);
  if (size > sh->best) {
    for (int32_t i = 0; i < size; i++) sh->H[i] = sh->orig[w->C[i]];
    __atomic_store_n(&sh->best, size, __ATOMIC_RELEASE);
  }
  pthread_mutex_unlock(&sh->mu);
}

/* Branch(C, P) with |C| = csize, P = idx[0..cnt) in natural order with
 * their colours; the incumbent is re-read before every test */
static void th_branch(th_worker *w, int32_t csize, int32_t *idx, int32_t *colors, int32_t cnt) {
  w->nodes++;
  int32_t *pidx = (int32_t *)malloc(((size_t)cnt + 1) * sizeof(int32_t));
  int32_t *pcol = (int32_t *)malloc(((size_t)cnt + 1) * sizeof(int32_t));
  int32_t *scr = (int32_t *)malloc(((size_t)cnt + 3) * sizeof(int32_t));
  if (!pidx || !pcol || !scr) { w->err = ORC_ERR_OOM; free(pidx); free(pcol); free(scr); return; }
  while (cnt > 0 && cnt + csize > th_best(w)) {
    int32_t at = 0;
    for (int32_t i = 1; i < cnt; i++) if (colors[i] >= colors[at]) at = i;
    int32_t u = idx[at], cu = colors[at];
    for (int32_t i = at; i + 1 < cnt; i++) { idx[i] = idx[i + 1]; colors[i] = colors[i + 1]; }
    cnt--;
    if (csize + cu <= th_best(w)) break;
    w->C[csize] = w->P[u];
    int32_t c2 = csize + 1;
    int32_t np2 = 0;
    for (int32_t i = 0; i < cnt; i++)
      if (w->adj[(int64_t)u * w->np + idx[i]]) pidx[np2++] = idx[i];
    if (np2 > 0) {
      int32_t L = th_color_list(w, pidx, np2, pcol, scr);
      if (c2 + L > th_best(w)) {
        th_branch(w, c2, pidx, pcol, np2);
        if (w->err) break;
      }
    } else if (c2 > th_best(w)) {
      th_raise(w, c2);
    }
  }
  free(pidx); free(pcol); free(scr);
}

static int cmp_knkey_id(const void *x, const void *y) {
  const knkey *a = (const knkey *)x, *b = (const knkey *)y;
  return (a->id > b->id) - (a->id < b->id);
}

/* the search rooted at u (new id): cliques whose lowest-ranked member is u */
static void th_root(th_worker *w, int32_t u, int32_t *kn, uint8_t *in, int32_t *idx, int32_t *col, int32_t *scr,
                    knkey *ord, int32_t *nat, int32_t *ncol) {
  th_search *sh = w->sh;
  if (sh->opos[u] % sh->part_count != sh->part_rank) return; /* another part's root */
  int32_t h = th_best(w);
  if (sh->K[u] < h) return; /* K(u) + 1 <= |H| */
  w->ib_calls++;
  int32_t np = 0;
  for (int64_t e = sh->orp[u]; e < sh->orp[u + 1]; e++)
    if (sh->K[sh->oci[e]] >= h) w->P[np++] = sh->oci[e];
  if (np + 1 <= h) return;
  w->ib_full++;
  w->np = np;
  /* G[P]: each pair {a, b} of P appears in the later-neighbour list of the
   * one of lower rank */
  for (int32_t a = 0; a < np; a++) w->mark[w->P[a]] = a + 1;
  memset(w->adj, 0, (size_t)np * (size_t)np);
  for (int32_t a = 0; a < np; a++) {
    int32_t x = w->P[a];
    for (int64_t e = sh->orp[x]; e < sh->orp[x + 1]; e++) {
      int32_t b = w->mark[sh->oci[e]];
      if (b) {
        w->adj[(int64_t)a * np + (b - 1)] = 1;
        w->adj[(int64_t)(b - 1) * np + a] = 1;
      }
    }
  }
  for (int32_t a = 0; a < np; a++) w->mark[w->P[a]] = 0;
  for (int32_t a = 0; a < np; a++) in[a] = 1;
  small_cores(w->adj, np, in, kn);
  h = th_best(w);
  int32_t cnt = 0;
  for (int32_t a = 0; a < np; a++)
    if (kn[a] + 1 >= h) { ord[cnt].i = a; ord[cnt].kn = kn[a]; ord[cnt].id = sh->orig[w->P[a]]; cnt++; }
  if (cnt + 1 <= h) return;
  qsort(ord, (size_t)cnt, sizeof(knkey), cmp_knkey);
  for (int32_t j = 0; j < cnt; j++) idx[j] = ord[j].i;
  int32_t L = th_color_list(w, idx, cnt, col, scr);
  if (1 + L <= th_best(w)) return;
  /* Branch({u}, kept) with the kept vertices in natural order: increasing
   * original vertex id, as in orc_max_clique (the recolouring order of
   * Branch is free; ascending rank, the peel order, colours worst) */
  for (int32_t j = 0; j < cnt; j++) { ord[j].i = idx[j]; ord[j].kn = col[j]; ord[j].id = sh->orig[w->P[idx[j]]]; }
  qsort(ord, (size_t)cnt, sizeof(knkey), cmp_knkey_id);
  int32_t c = 0;
  for (int32_t j = 0; j < cnt; j++) { nat[c] = ord[j].i; ncol[c] = ord[j].kn; c++; }
  w->C[0] = u;
  th_branch(w, 1, nat, ncol, c);
}

static void *search_worker(void *arg) {
  th_worker *w = (th_worker *)arg;
  th_search *sh = w->sh;
  size_t kp = (size_t)sh->kmax + 2;
  int32_t *kn = (int32_t *)malloc(kp * sizeof(int32_t));
  uint8_t *in = (uint8_t *)malloc(kp);
  int32_t *idx = (int32_t *)malloc(kp * sizeof(int32_t));
  int32_t *col = (int32_t *)malloc(kp * sizeof(int32_t));
  int32_t *scr = (int32_t *)malloc((kp + 3) * sizeof(int32_t));
  knkey *ord = (knkey *)malloc(kp * sizeof(knkey));
  int32_t *nat = (int32_t *)malloc(kp * sizeof(int32_t));
  int32_t *ncol = (int32_t *)malloc(kp * sizeof(int32_t));
  if (!kn || !in || !idx || !col || !scr || !ord || !nat || !ncol) {
    w->err = ORC_ERR_OOM;
  } else {
    for (;;) {
      int64_t i = __atomic_fetch_add(&sh->next, 1, __ATOMIC_RELAXED);
      if (i >= sh->n2) break;
      th_root(w, (int32_t)i, kn, in, idx, col, scr, ord, nat, ncol);
      if (w->err) break;
    }
  }
  free(kn); free(in); free(idx); free(col); free(scr); free(ord); free(nat); free(ncol);
  pthread_mutex_lock(&sh->mu);
  sh->ib_calls += w->ib_calls;
  sh->ib_full += w->ib_full;
  sh->nodes += w->nodes;
  if (w->err) sh->err = w->err;
  pthread_mutex_unlock(&sh->mu);
  return NULL;
}

static int run_threads(int threads, void *(*fn)(void *), void *args, size_t stride) {
  pthread_t *th = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
  if (!th) return ORC_ERR_OOM;
  int started = 0, rc = ORC_OK;
  for (int t = 0; t < threads; t++) {
    if (pthread_create(&th[t], NULL, fn, (char *)args + (size_t)t * stride) != 0) { rc = ORC_ERR_OOM; break; }
    started++;
  }
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  free(th);
  return rc;
}

/* A degeneracy order: every vertex has at most K(v) neighbours after it. */
static int is_degeneracy_order(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *K, const int32_t *order,
                               int32_t *pos) {
  for (int64_t i = 0; i < n; i++) pos[i] = -1;
  for (int64_t i = 0; i < n; i++) {
    if (order[i] < 0 || order[i] >= n || pos[order[i]] >= 0) return 0;
    pos[order[i]] = (int32_t)i;
  }
  for (int64_t v = 0; v < n; v++) {
    int64_t later = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) later += pos[ci[e]] > pos[v];
    if (later > K[v]) return 0;
  }
  return 1;
}

static int max_clique_part(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *order_in,
                           int32_t part_rank, int32_t part_count, int32_t threads, int32_t *omega_out,
                           int32_t *witness, int32_t cap, orc_stats *st);

int orc_max_clique_threads(int64_t n, const int64_t *rp, const int32_t *ci, int32_t threads, int32_t *omega_out,
                           int32_t *witness, int32_t cap, orc_stats *st) {
  return max_clique_part(n, rp, ci, NULL, 0, 1, threads, omega_out, witness, cap, st);
}

/* The threaded search over the roots at positions part_rank, part_rank +
 * part_count, ... of `order` (a degeneracy order of the graph; NULL = the
 * Batagelj-Zaversnik order).  omega_out and witness: the largest clique
 * this part found, which is the heuristic's clique when no root of the part
 * beats it; the maximum over all parts is omega(G), since every clique has
 * exactly one lowest-ranked member.  ORC_ERR_ARG if order is not a
 * degeneracy order. */
int orc_max_clique_part(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *order, int32_t part_rank,
                        int32_t part_count, int32_t threads, int32_t *omega_out, int32_t *witness, int32_t cap,
                        orc_stats *st) {
  if (part_count < 1 || part_rank < 0 || part_rank >= part_count) return ORC_ERR_ARG;
  return max_clique_part(n, rp, ci, order, part_rank, part_count, threads, omega_out, witness, cap, st);
}

static int max_clique_part(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *order_in,
                           int32_t part_rank, int32_t part_count, int32_t threads, int32_t *omega_out,
                           int32_t *witness, int32_t cap, orc_stats *st) {
  if (n < 0 || threads < 1 || threads > 1024) return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  *omega_out = 0;
  if (n == 0) return ORC_OK;
  int rc = ORC_OK;
  int32_t *K0 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  vkey *hord = (vkey *)malloc((size_t)n * sizeof(vkey));
  int32_t *newid = NULL, *orig = NULL, *K2 = NULL, *oci = NULL, *H = NULL, *opos = NULL, *fpos = NULL;
  int64_t *orp = NULL;
  th_worker *wk = NULL;
  th_heur hh;
  th_search sh;
  memset(&hh, 0, sizeof(hh));
  memset(&sh, 0, sizeof(sh));
  pthread_mutex_init(&hh.mu, NULL);
  pthread_mutex_init(&sh.mu, NULL);
  if (!K0 || !order || !hord) { rc = ORC_ERR_OOM; goto out; }
  /* 1. core numbers and the degeneracy order (the given one if any) */
  if ((rc = orc_core_numbers(n, rp, ci, K0, order)) != ORC_OK) goto out;
  fpos = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!fpos) { rc = ORC_ERR_OOM; goto out; }
  if (order_in) {
    if (!is_degeneracy_order(n, rp, ci, K0, order_in, fpos)) { rc = ORC_ERR_ARG; goto out; }
    memcpy(order, order_in, (size_t)n * sizeof(int32_t));
  }
  for (int64_t i = 0; i < n; i++) fpos[order[i]] = (int32_t)i;
  int32_t kmax = 0;
  int64_t maxd = 0;
  for (int64_t v = 0; v < n; v++) {
    if (K0[v] > kmax) kmax = K0[v];
    if (rp[v + 1] - rp[v] > maxd) maxd = rp[v + 1] - rp[v];
  }
  st->max_core = kmax;
  H = (int32_t *)malloc(((size_t)kmax + 2) * sizeof(int32_t));
  if (!H) { rc = ORC_ERR_OOM; goto out; }
  /* 2. Algorithm 1, printed form, shared running maximum */
  for (int64_t v = 0; v < n; v++) { hord[v].v = (int32_t)v; hord[v].k = K0[v]; hord[v].d = rp[v + 1] - rp[v]; }
  qsort(hord, (size_t)n, sizeof(vkey), cmp_vkey);
  hh.n = n; hh.rp = rp; hh.ci = ci; hh.core = K0; hh.ord = hord; hh.maxd = maxd; hh.best = H;
  /* every worker gets the same shared record (stride 0) */
  if ((rc = run_threads(threads, heur_worker, &hh, 0)) != ORC_OK) goto out;
  if (hh.err) { rc = hh.err; goto out; }
  free(hord); hord = NULL;
  int32_t hs = hh.max;
  st->heuristic = hs;
  /* 3. explicit pruning; new ids in degeneracy order, later neighbours only */
  newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!newid) { rc = ORC_ERR_OOM; goto out; }
  int64_t n2 = 0;
  for (int64_t v = 0; v < n; v++) newid[v] = -1;
  for (int64_t i = 0; i < n; i++) if (K0[order[i]] >= hs) newid[order[i]] = (int32_t)n2++;
  st->pruned_n = n2;
  orp = (int64_t *)malloc(((size_t)n2 + 1) * sizeof(int64_t));
  orig = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  K2 = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  opos = (int32_t *)malloc(((size_t)n2 + 1) * sizeof(int32_t));
  if (!orp || !orig || !K2 || !opos) { rc = ORC_ERR_OOM; goto out; }
  orp[0] = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = order[i];
    if (newid[v] < 0) continue;
    int64_t d = 0;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) if (newid[ci[e]] > newid[v]) d++;
    orig[newid[v]] = v;
    K2[newid[v]] = K0[v];
    opos[newid[v]] = fpos[v];
    orp[newid[v] + 1] = orp[newid[v]] + d;
  }
  oci = (int32_t *)malloc(((size_t)orp[n2] + 1) * sizeof(int32_t));
  if (!oci) { rc = ORC_ERR_OOM; goto out; }
  for (int64_t i = 0; i < n; i++) {
    int32_t v = order[i];
    if (newid[v] < 0) continue;
    int64_t o = orp[newid[v]];
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) if (newid[ci[e]] > newid[v]) oci[o++] = newid[ci[e]];
    qsort(oci + orp[newid[v]], (size_t)(o - orp[newid[v]]), sizeof(int32_t), cmp_i32_asc);
  }
  free(newid); newid = NULL;
  /* 4. the roots, shared by the workers */
  sh.n2 = n2; sh.orp = orp; sh.oci = oci; sh.K = K2; sh.orig = orig; sh.kmax = kmax;
  sh.best = hs; sh.H = H;
  sh.opos = opos; sh.part_rank = part_rank; sh.part_count = part_count;
  wk = (th_worker *)calloc((size_t)threads, sizeof(th_worker));
  if (!wk) { rc = ORC_ERR_OOM; goto out; }
  for (int t = 0; t < threads; t++) {
    wk[t].sh = &sh;
    wk[t].mark = (int32_t *)calloc((size_t)n2 + 1, sizeof(int32_t));
    wk[t].P = (int32_t *)malloc(((size_t)kmax + 2) * sizeof(int32_t));
    wk[t].C = (int32_t *)malloc(((size_t)kmax + 2) * sizeof(int32_t));
    wk[t].adj = (uint8_t *)malloc(((size_t)kmax + 2) * ((size_t)kmax + 2));
    if (!wk[t].mark || !wk[t].P || !wk[t].C || !wk[t].adj) { rc = ORC_ERR_OOM; goto out; }
  }
  if ((rc = run_threads(threads, search_worker, wk, sizeof(th_worker))) != ORC_OK) goto out;
  if (sh.err) { rc = sh.err; goto out; }
  st->initial_branch = sh.ib_calls;
  st->full_branch = sh.ib_full;
  st->nodes = sh.nodes;
  *omega_out = sh.best;
  if (sh.best > cap) rc = ORC_ERR_BUFFER;
  else {
    qsort(H, (size_t)sh.best, sizeof(int32_t), cmp_i32_asc);
    memcpy(witness, H, (size_t)sh.best * sizeof(int32_t));
  }
out:
  if (wk)
    for (int t = 0; t < threads; t++) { free(wk[t].mark); free(wk[t].P); free(wk[t].C); free(wk[t].adj); }
  free(wk);
  free(K0); free(order); free(hord); free(newid); free(orig); free(K2); free(oci); free(orp); free(H);
  free(opos); free(fpos);
  pthread_mutex_destroy(&hh.mu);
  pthread_mutex_destroy(&sh.mu);
  return rc;
}
