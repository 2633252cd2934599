/*
 * CPU oracle for dynamic-graph PageRank: plain, single-threaded, FP64.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header, table or helper with the
 * CUDA library, and it is written for reading against the paper, not for
 * speed: sorting is qsort, membership is bsearch, every loop is in the
 * paper's order.
 *
 * What it computes (arXiv 2407.19562, "Lock-Free Computation of PageRank in
 * Dynamic Graphs"):
 *   - graph model: a set of directed edges; CSR (out-rows) and CSC (in-rows)
 *     with sorted unique rows; optional self-loop on every vertex (Sec. 5.1.3
 *     removes dead ends this way, Sec. 5.1.4 re-adds them with each batch);
 *   - batch update (Sec. 3.4): G^t = (G^{t-1} minus deletions) plus
 *     insertions, deletions taken first; the real changes are
 *     Delta- = E^{t-1} \ E^t and Delta+ = E^t \ E^{t-1};
 *   - Static_BB (Alg. 3) and ND_BB (Alg. 5): Jacobi power iteration of Eq. 1;
 *   - Static_LF (Alg. 4) and ND_LF (Alg. 6), run on one thread;
 *   - DF_BB (Alg. 1) with marks taking effect from the next iteration;
 *   - DF_LF (Alg. 2) run on one thread, vertices visited in ascending id;
 *   - the initial affected set of the DF approach (Sec. 4.1);
 *   - sampled rows of an updated graph straight from raw edges, for checks
 *     at sizes where the whole model is too slow.
 *
 * Parity pins (what fixes each function independently of this file) are in
 * the tests: closed forms, a dense linear solve, brute force on adjacency
 * matrices, the worked example of Sec. 4.1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

typedef struct orc_graph {
  int32_t n;
  int64_t m;
  int self_loops;
  int64_t* out_off; /* n + 1 */
  int32_t* out_idx; /* m, row u holds the targets of u's out-edges, ascending */
  int64_t* in_off;  /* n + 1 */
  int32_t* in_idx;  /* m, row v holds the sources of v's in-edges, ascending */
  /* Real changes of the batch that produced this snapshot, sorted by (src, dst). */
  int64_t n_del, n_ins;
  uint64_t* del_keys; /* src << 32 | dst */
  uint64_t* ins_keys;
} orc_graph;

typedef struct orc_stats {
  int64_t iterations; /* iterations (BB) or passes (LF) executed */
  int64_t processed;  /* vertex rank computations */
  int64_t edges;      /* in-edges gathered */
  double last_delta;  /* BB: last L-inf iterate difference */
  int32_t converged;  /* 1 if the stopping test passed before MAX_ITERATIONS */
  int32_t affected;   /* vertices marked affected at exit (DF) */
} orc_stats;

int orc_version(void) { return 1; }

/* ----------------------------------------------------------------------- */
/* Graph model                                                              */
/* ----------------------------------------------------------------------- */

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

static inline uint64_t key_of(int32_t u, int32_t v) {
  return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
}
static inline int32_t key_hi(uint64_t k) { return (int32_t)(k >> 32); }
static inline int32_t key_lo(uint64_t k) { return (int32_t)(k & 0xFFFFFFFFu); }

static int64_t sort_unique(uint64_t* k, int64_t m) {
  if (m <= 0) return 0;
  qsort(k, (size_t)m, sizeof(uint64_t), cmp_u64);
  int64_t w = 1;
  for (int64_t i = 1; i < m; ++i)
    if (k[i] != k[w - 1]) k[w++] = k[i];
  return w;
}

static int has_key(const uint64_t* k, int64_t m, uint64_t x) {
  return m > 0 && bsearch(&x, k, (size_t)m, sizeof(uint64_t), cmp_u64) != NULL;
}

void orc_graph_free(orc_graph* g) {
  if (!g) return;
  free(g->out_off); free(g->out_idx); free(g->in_off); free(g->in_idx);
  free(g->del_keys); free(g->ins_keys);
  free(g);
}

/* Fills CSR and CSC from a sorted unique key array (src << 32 | dst). */
static int fill_from_keys(orc_graph* g, const uint64_t* keys, int64_t m) {
  int32_t n = g->n;
  g->m = m;
  g->out_off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->in_off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->out_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  g->in_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  uint64_t* t = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
  if (!g->out_off || !g->in_off || !g->out_idx || !g->in_idx || !t) { free(t); return ORC_ENOMEM; }
  for (int64_t i = 0; i < m; ++i) {
    g->out_off[key_hi(keys[i]) + 1]++;
    g->out_idx[i] = key_lo(keys[i]);
    t[i] = key_of(key_lo(keys[i]), key_hi(keys[i]));
  }
  for (int32_t v = 0; v < n; ++v) g->out_off[v + 1] += g->out_off[v];
  qsort(t, (size_t)m, sizeof(uint64_t), cmp_u64);
  for (int64_t i = 0; i < m; ++i) {
    g->in_off[key_hi(t[i]) + 1]++;
    g->in_idx[i] = key_lo(t[i]);
  }
  for (int32_t v = 0; v < n; ++v) g->in_off[v + 1] += g->in_off[v];
  free(t);
  return ORC_OK;
}

/*
 * Builds the snapshot G^0 from m raw edges (duplicates allowed). With
 * self_loops != 0 every vertex gets the edge (v, v), as Sec. 5.1.3 does to
 * remove dead ends. Ids must lie in [0, n).
 */
int orc_graph_build(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                    int self_loops, orc_graph** out) {
  if (n <= 0 || m_raw < 0 || !out) return ORC_EINVAL;
  *out = NULL;
  int64_t cap = m_raw + (self_loops ? n : 0);
  uint64_t* k = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
  if (!k) return ORC_ENOMEM;
  int64_t c = 0;
  for (int64_t i = 0; i < m_raw; ++i) {
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) { free(k); return ORC_EINVAL; }
    k[c++] = key_of(src[i], dst[i]);
  }
  if (self_loops)
    for (int32_t v = 0; v < n; ++v) k[c++] = key_of(v, v);
  c = sort_unique(k, c);
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  if (!g) { free(k); return ORC_ENOMEM; }
  g->n = n;
  g->self_loops = self_loops ? 1 : 0;
  int rc = fill_from_keys(g, k, c);
  free(k);
  if (rc != ORC_OK) { orc_graph_free(g); return rc; }
  *out = g;
  return ORC_OK;
}

/*
 * Applies a batch (Sec. 3.4): deletions first, then insertions. Duplicate
 * entries collapse; deleting an absent edge, inserting a present edge and
 * (with self-loops on) deleting a self-loop change nothing. The returned
 * snapshot records the real changes Delta- = E^{t-1} \ E^t and
 * Delta+ = E^t \ E^{t-1}, sorted by (src, dst).
 */
int orc_graph_apply(const orc_graph* g, int64_t n_del, const int32_t* del_src,
                    const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                    const int32_t* ins_dst, orc_graph** out, int64_t* n_real) {
  if (!g || !out || n_del < 0 || n_ins < 0) return ORC_EINVAL;
  *out = NULL;
  int32_t n = g->n;
  for (int64_t i = 0; i < n_del; ++i)
    if (del_src[i] < 0 || del_src[i] >= n || del_dst[i] < 0 || del_dst[i] >= n) return ORC_EINVAL;
  for (int64_t i = 0; i < n_ins; ++i)
    if (ins_src[i] < 0 || ins_src[i] >= n || ins_dst[i] < 0 || ins_dst[i] >= n) return ORC_EINVAL;

  /* Previous edge set as sorted keys (CSR order is already sorted). */
  uint64_t* old_k = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(g->m > 0 ? g->m : 1));
  uint64_t* dk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_del > 0 ? n_del : 1));
  uint64_t* ik = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_ins > 0 ? n_ins : 1));
  if (!old_k || !dk || !ik) { free(old_k); free(dk); free(ik); return ORC_ENOMEM; }
  for (int32_t u = 0; u < n; ++u)
    for (int64_t e = g->out_off[u]; e < g->out_off[u + 1]; ++e) old_k[e] = key_of(u, g->out_idx[e]);
  for (int64_t i = 0; i < n_del; ++i) dk[i] = key_of(del_src[i], del_dst[i]);
  for (int64_t i = 0; i < n_ins; ++i) ik[i] = key_of(ins_src[i], ins_dst[i]);
  int64_t nd = sort_unique(dk, n_del), ni = sort_unique(ik, n_ins);

  /* Real deletions: present before, not a protected self-loop, not re-inserted. */
  int64_t rd = 0;
  for (int64_t i = 0; i < nd; ++i) {
    uint64_t x = dk[i];
    if (g->self_loops && key_hi(x) == key_lo(x)) continue;
    if (!has_key(old_k, g->m, x)) continue;
    if (has_key(ik, ni, x)) continue;
    dk[rd++] = x;
  }
  /* Real insertions: absent before. */
  int64_t ri = 0;
  for (int64_t i = 0; i < ni; ++i)
    if (!has_key(old_k, g->m, ik[i])) ik[ri++] = ik[i];

  int64_t new_m = g->m - rd + ri;
  uint64_t* nk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(new_m > 0 ? new_m : 1));
  if (!nk) { free(old_k); free(dk); free(ik); return ORC_ENOMEM; }
  int64_t c = 0;
  for (int64_t e = 0; e < g->m; ++e)
    if (!has_key(dk, rd, old_k[e])) nk[c++] = old_k[e];
  for (int64_t i = 0; i < ri; ++i) nk[c++] = ik[i];
  qsort(nk, (size_t)c, sizeof(uint64_t), cmp_u64);
  free(old_k);

  orc_graph* h = (orc_graph*)calloc(1, sizeof(orc_graph));
  if (!h) { free(nk); free(dk); free(ik); return ORC_ENOMEM; }
  h->n = n;
  h->self_loops = g->self_loops;
  int rc = fill_from_keys(h, nk, c);
  free(nk);
  h->n_del = rd; h->n_ins = ri;
  h->del_keys = dk; h->ins_keys = ik;
  if (rc != ORC_OK) { orc_graph_free(h); return rc; }
  if (n_real) { n_real[0] = rd; n_real[1] = ri; }
  *out = h;
  return ORC_OK;
}

int32_t orc_graph_n(const orc_graph* g) { return g->n; }
int64_t orc_graph_m(const orc_graph* g) { return g->m; }

/* Copies CSR and CSC out (any pointer may be NULL). */
void orc_graph_export(const orc_graph* g, int64_t* out_off, int32_t* out_idx, int64_t* in_off,
                      int32_t* in_idx) {
  size_t n1 = (size_t)g->n + 1, m = (size_t)g->m;
  if (out_off) memcpy(out_off, g->out_off, n1 * sizeof(int64_t));
  if (out_idx) memcpy(out_idx, g->out_idx, m * sizeof(int32_t));
  if (in_off) memcpy(in_off, g->in_off, n1 * sizeof(int64_t));
  if (in_idx) memcpy(in_idx, g->in_idx, m * sizeof(int32_t));
}

/* Copies the real changes of the last batch out as (src, dst) pairs. */
void orc_graph_last_batch(const orc_graph* g, int64_t* counts, int32_t* del_src, int32_t* del_dst,
                          int32_t* ins_src, int32_t* ins_dst) {
  if (counts) { counts[0] = g->n_del; counts[1] = g->n_ins; }
  for (int64_t i = 0; del_src && i < g->n_del; ++i) {
    del_src[i] = key_hi(g->del_keys[i]); del_dst[i] = key_lo(g->del_keys[i]);
  }
  for (int64_t i = 0; ins_src && i < g->n_ins; ++i) {
    ins_src[i] = key_hi(g->ins_keys[i]); ins_dst[i] = key_lo(g->ins_keys[i]);
  }
}

/* ----------------------------------------------------------------------- */
/* PageRank of one vertex, Eq. 1                                            */
/* ----------------------------------------------------------------------- */

static inline int64_t outdeg(const orc_graph* g, int32_t u) {
  return g->out_off[u + 1] - g->out_off[u];
}

/* Sum over dead ends (no out-edges) of R, for the teleport reading. */
static double dangling_mass(const orc_graph* g, const double* R) {
  double d = 0.0;
  for (int32_t u = 0; u < g->n; ++u)
    if (outdeg(g, u) == 0) d += R[u];
  return d;
}

/*
 * Eq. 1: R[v] = alpha * sum_{u in in(v)} R[u] / |out(u)| + (1 - alpha) / n,
 * accumulated term by term as the algorithms print it: r starts at
 * (1 - alpha) / n and each in-neighbour adds alpha * R[u] / |out(u)|.
 * With dead_end == 1 (teleport reading, not in the paper's experiments)
 * alpha * D / n is added, D the rank held by dead ends.
 */
static double rank_of(const orc_graph* g, const double* R, int32_t v, double alpha, double D,
                      int dead_end, orc_stats* st) {
  double r = (1.0 - alpha) / (double)g->n;
  for (int64_t e = g->in_off[v]; e < g->in_off[v + 1]; ++e) {
    int32_t u = g->in_idx[e];
    r = r + alpha * R[u] / (double)outdeg(g, u);
  }
  if (dead_end) r = r + alpha * D / (double)g->n;
  if (st) { st->processed++; st->edges += g->in_off[v + 1] - g->in_off[v]; }
  return r;
}

/* ----------------------------------------------------------------------- */
/* Static_BB (Alg. 3) / ND_BB (Alg. 5)                                      */
/* ----------------------------------------------------------------------- */

/*
 * Jacobi power iteration with two vectors. R_init == NULL starts from 1/n
 * (Static_BB, Alg. 3); otherwise from R_init (ND_BB, Alg. 5). Each iteration
 * computes every vertex from the previous vector, takes the L-inf difference,
 * swaps, and stops when the difference is <= tol or after max_iter
 * iterations. The paper's reference ranks (Sec. 5.1.5) are this with
 * tol = 1e-100 and max_iter = 500.
 */
int orc_static_bb(const orc_graph* g, const double* R_init, double alpha, double tol,
                  int max_iter, int dead_end, double* R_out, orc_stats* st) {
  if (!g || !R_out || max_iter < 0) return ORC_EINVAL;
  int32_t n = g->n;
  double* R = (double*)malloc(sizeof(double) * (size_t)n);
  double* Rn = (double*)malloc(sizeof(double) * (size_t)n);
  if (!R || !Rn) { free(R); free(Rn); return ORC_ENOMEM; }
  orc_stats s;
  memset(&s, 0, sizeof s);
  for (int32_t v = 0; v < n; ++v) R[v] = R_init ? R_init[v] : 1.0 / (double)n;
  memcpy(Rn, R, sizeof(double) * (size_t)n);
  for (int i = 0; i < max_iter; ++i) {
    double D = dead_end ? dangling_mass(g, R) : 0.0;
    for (int32_t v = 0; v < n; ++v) Rn[v] = rank_of(g, R, v, alpha, D, dead_end, &s);
    double dR = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double d = fabs(Rn[v] - R[v]);
      if (d > dR) dR = d;
    }
    double* t = R; R = Rn; Rn = t;
    s.iterations = i + 1;
    s.last_delta = dR;
    if (dR <= tol) { s.converged = 1; break; }
  }
  memcpy(R_out, R, sizeof(double) * (size_t)n);
  free(R); free(Rn);
  if (st) *st = s;
  return ORC_OK;
}

/* ----------------------------------------------------------------------- */
/* Static_LF (Alg. 4) / ND_LF (Alg. 6) on one thread                        */
/* ----------------------------------------------------------------------- */

/*
 * Asynchronous (in-place) iteration with per-vertex not-converged flags R_C.
 * R_C starts at 1 for every vertex: the text of the appendix says no vertex
 * has converged at the start, and R_C = 1 means not converged (Sec. 4.3),
 * so the printed initialisation to 0 is read as a typo. A pass visits all
 * vertices in ascending id; R_C[v] is cleared when v's change is <= tol;
 * the iteration stops after a pass that leaves every flag clear.
 */
int orc_static_lf(const orc_graph* g, const double* R_init, double alpha, double tol,
                  int max_iter, double* R_out, orc_stats* st) {
  if (!g || !R_out || max_iter < 0) return ORC_EINVAL;
  int32_t n = g->n;
  uint8_t* RC = (uint8_t*)malloc((size_t)n);
  if (!RC) return ORC_ENOMEM;
  orc_stats s;
  memset(&s, 0, sizeof s);
  for (int32_t v = 0; v < n; ++v) { R_out[v] = R_init ? R_init[v] : 1.0 / (double)n; RC[v] = 1; }
  for (int i = 0; i < max_iter; ++i) {
    for (int32_t v = 0; v < n; ++v) {
      double r = rank_of(g, R_out, v, alpha, 0.0, 0, &s);
      double dr = fabs(r - R_out[v]);
      R_out[v] = r;
      if (dr <= tol && RC[v] == 1) RC[v] = 0;
    }
    s.iterations = i + 1;
    int all = 1;
    for (int32_t v = 0; v < n && all; ++v) all = (RC[v] == 0);
    if (all) { s.converged = 1; break; }
  }
  free(RC);
  if (st) *st = s;
  return ORC_OK;
}

/* ----------------------------------------------------------------------- */
/* Dynamic Frontier                                                         */
/* ----------------------------------------------------------------------- */

/*
 * Initial marking of the DF approach (Sec. 4.1; Alg. 1 and Alg. 2 marking
 * loops): for every edge (u, v) of Delta- or Delta+, every out-neighbour of u
 * in G^{t-1} or G^t is affected. out_{t-1}(u) union out_t(u) equals out_t(u)
 * plus the targets of u's deleted edges, because Delta- = E^{t-1} \ E^t and
 * Delta+ = E^t \ E^{t-1}; so G^t and its recorded batch suffice.
 * With self-loops, u is its own out-neighbour and is marked too.
 * mark_u(u) is called once per distinct source.
 */
static void mark_initial(const orc_graph* gt, uint8_t* VA, uint8_t* RC, uint8_t* C) {
  for (int pass = 0; pass < 2; ++pass) {
    int64_t cnt = pass == 0 ? gt->n_del : gt->n_ins;
    const uint64_t* ks = pass == 0 ? gt->del_keys : gt->ins_keys;
    for (int64_t i = 0; i < cnt; ++i) {
      int32_t u = key_hi(ks[i]);
      if (C && C[u]) continue;                  /* source already checked */
      for (int64_t e = gt->out_off[u]; e < gt->out_off[u + 1]; ++e) {
        VA[gt->out_idx[e]] = 1;
        if (RC) RC[gt->out_idx[e]] = 1;
      }
      /* targets of u's deleted edges: del_keys is sorted by (src, dst), so
       * they form one run starting at the first key >= (u, 0) */
      int64_t lo = 0, hi = gt->n_del;
      while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (gt->del_keys[mid] < key_of(u, 0)) lo = mid + 1; else hi = mid;
      }
      for (int64_t j = lo; j < gt->n_del && key_hi(gt->del_keys[j]) == u; ++j) {
        VA[key_lo(gt->del_keys[j])] = 1;
        if (RC) RC[key_lo(gt->del_keys[j])] = 1;
      }
      if (C) C[u] = 1;
    }
  }
}

int orc_initial_affected(const orc_graph* gt, uint8_t* VA) {
  if (!gt || !VA) return ORC_EINVAL;
  memset(VA, 0, (size_t)gt->n);
  uint8_t* C = (uint8_t*)calloc((size_t)gt->n, 1);
  if (!C) return ORC_ENOMEM;
  mark_initial(gt, VA, NULL, C);
  free(C);
  return ORC_OK;
}

/*
 * DF_BB (Alg. 1): Jacobi iteration restricted to affected vertices. Marks
 * made while computing iteration i take effect from iteration i + 1 (the
 * algorithm leaves this to thread timing; this reading makes the result
 * deterministic). A vertex whose change exceeds tol_f marks its out-neighbours
 * in G^t. The iteration stops when the L-inf difference of consecutive
 * iterates is <= tol, or after max_iter iterations.
 * If VA_trace != NULL, VA_trace[k * n + v] receives the affected flags in
 * force during iteration k, for k < trace_len (k = 0 is the initial marking).
 */
int orc_df_bb(const orc_graph* gt, const double* R_prev, double alpha, double tol, double tol_f,
              int max_iter, double* R_out, orc_stats* st, uint8_t* VA_trace, int trace_len) {
  if (!gt || !R_prev || !R_out || max_iter < 0) return ORC_EINVAL;
  int32_t n = gt->n;
  double* R = (double*)malloc(sizeof(double) * (size_t)n);
  double* Rn = (double*)malloc(sizeof(double) * (size_t)n);
  uint8_t* VA = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* VAn = (uint8_t*)calloc((size_t)n, 1);
  if (!R || !Rn || !VA || !VAn) { free(R); free(Rn); free(VA); free(VAn); return ORC_ENOMEM; }
  orc_stats s;
  memset(&s, 0, sizeof s);
  memcpy(R, R_prev, sizeof(double) * (size_t)n);
  memcpy(Rn, R_prev, sizeof(double) * (size_t)n);
  mark_initial(gt, VA, NULL, NULL);
  for (int i = 0; i < max_iter; ++i) {
    if (VA_trace && i < trace_len) memcpy(VA_trace + (size_t)i * n, VA, (size_t)n);
    memcpy(VAn, VA, (size_t)n);
    for (int32_t v = 0; v < n; ++v) {
      if (!VA[v]) continue;
      double r = rank_of(gt, R, v, alpha, 0.0, 0, &s);
      double dr = fabs(r - R[v]);
      Rn[v] = r;
      if (dr > tol_f)
        for (int64_t e = gt->out_off[v]; e < gt->out_off[v + 1]; ++e) VAn[gt->out_idx[e]] = 1;
    }
    double dR = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double d = fabs(Rn[v] - R[v]);
      if (d > dR) dR = d;
    }
    double* t = R; R = Rn; Rn = t;
    memcpy(VA, VAn, (size_t)n);
    s.iterations = i + 1;
    s.last_delta = dR;
    if (dR <= tol) { s.converged = 1; break; }
  }
  if (VA_trace)
    for (int k = (int)s.iterations; k < trace_len; ++k) memcpy(VA_trace + (size_t)k * n, VA, (size_t)n);
  int32_t a = 0;
  for (int32_t v = 0; v < n; ++v) a += VA[v];
  s.affected = a;
  memcpy(R_out, R, sizeof(double) * (size_t)n);
  free(R); free(Rn); free(VA); free(VAn);
  if (st) *st = s;
  return ORC_OK;
}

/*
 * Dead-end mass D = sum of R[u] over vertices u with no out-edges (the
 * teleport reading of Sec. 5.1.3).
 */
int orc_dangling_mass(const orc_graph* g, const double* R, double* D) {
  if (!g || !R || !D) return ORC_EINVAL;
  *D = dangling_mass(g, R);
  return ORC_OK;
}

/*
 * DF_BB (Alg. 1) with the teleport reading of dead ends (the paper's runs
 * add self-loops instead, Sec. 5.1.3, and give no formula for this case).
 * Every recomputed rank gets alpha * D / n, D the dead-end mass of the
 * current ranks, taken at the start of each iteration. A vertex outside the
 * affected set keeps a rank computed with an older D, so the frontier rule
 * is extended to the shared term: when alpha * |D - D_last| / n > tol_f,
 * every vertex is affected from this iteration on and D_last becomes D.
 * D_last starts at D_before, the dead-end mass of R_prev on G^{t-1} (the D
 * that R_prev was computed with), so a batch that moves rank into or out of
 * dead ends by more than that bound recomputes every vertex at once.
 * Otherwise the steps are those of orc_df_bb.
 */
int orc_df_bb_teleport(const orc_graph* gt, const double* R_prev, double D_before, double alpha,
                       double tol, double tol_f, int max_iter, double* R_out, orc_stats* st) {
  if (!gt || !R_prev || !R_out || max_iter < 0) return ORC_EINVAL;
  int32_t n = gt->n;
  double* R = (double*)malloc(sizeof(double) * (size_t)n);
  double* Rn = (double*)malloc(sizeof(double) * (size_t)n);
  uint8_t* VA = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* VAn = (uint8_t*)calloc((size_t)n, 1);
  if (!R || !Rn || !VA || !VAn) { free(R); free(Rn); free(VA); free(VAn); return ORC_ENOMEM; }
  orc_stats s;
  memset(&s, 0, sizeof s);
  memcpy(R, R_prev, sizeof(double) * (size_t)n);
  memcpy(Rn, R_prev, sizeof(double) * (size_t)n);
  mark_initial(gt, VA, NULL, NULL);
  double D_last = D_before;
  for (int i = 0; i < max_iter; ++i) {
    double D = dangling_mass(gt, R);
    if (alpha * fabs(D - D_last) / (double)n > tol_f) {
      for (int32_t v = 0; v < n; ++v) VA[v] = 1;
      D_last = D;
    }
    memcpy(VAn, VA, (size_t)n);
    for (int32_t v = 0; v < n; ++v) {
      if (!VA[v]) continue;
      double r = rank_of(gt, R, v, alpha, D, 1, &s);
      double dr = fabs(r - R[v]);
      Rn[v] = r;
      if (dr > tol_f)
        for (int64_t e = gt->out_off[v]; e < gt->out_off[v + 1]; ++e) VAn[gt->out_idx[e]] = 1;
    }
    double dR = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double d = fabs(Rn[v] - R[v]);
      if (d > dR) dR = d;
    }
    double* t = R; R = Rn; Rn = t;
    memcpy(VA, VAn, (size_t)n);
    s.iterations = i + 1;
    s.last_delta = dR;
    if (dR <= tol) { s.converged = 1; break; }
  }
  int32_t a = 0;
  for (int32_t v = 0; v < n; ++v) a += VA[v];
  s.affected = a;
  memcpy(R_out, R, sizeof(double) * (size_t)n);
  free(R); free(Rn); free(VA); free(VAn);
  if (st) *st = s;
  return ORC_OK;
}

/*
 * DF_LF (Alg. 2) on a single thread. The marking phase checks each source
 * once (flag C); then each pass visits the affected vertices in ascending id,
 * updating R in place. A vertex whose change exceeds tol_f marks its
 * out-neighbours affected and not converged (R_C = 1); a vertex whose change
 * is <= tol is marked converged (R_C = 0), in that order. A vertex marked
 * during a pass is visited in the same pass when its id is larger. The
 * iteration stops after a pass that leaves every R_C clear, or after max_iter
 * passes.
 */
int orc_df_lf(const orc_graph* gt, const double* R_prev, double alpha, double tol, double tol_f,
              int max_iter, double* R_out, orc_stats* st) {
  if (!gt || !R_prev || !R_out || max_iter < 0) return ORC_EINVAL;
  int32_t n = gt->n;
  uint8_t* VA = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* RC = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* C = (uint8_t*)calloc((size_t)n, 1);
  if (!VA || !RC || !C) { free(VA); free(RC); free(C); return ORC_ENOMEM; }
  orc_stats s;
  memset(&s, 0, sizeof s);
  memcpy(R_out, R_prev, sizeof(double) * (size_t)n);
  mark_initial(gt, VA, RC, C);
  for (int i = 0; i < max_iter; ++i) {
    for (int32_t v = 0; v < n; ++v) {
      if (!VA[v]) continue;
      double r = rank_of(gt, R_out, v, alpha, 0.0, 0, &s);
      double dr = fabs(r - R_out[v]);
      R_out[v] = r;
      if (dr > tol_f)
        for (int64_t e = gt->out_off[v]; e < gt->out_off[v + 1]; ++e) {
          VA[gt->out_idx[e]] = 1;
          RC[gt->out_idx[e]] = 1;
        }
      if (dr <= tol) RC[v] = 0;
    }
    s.iterations = i + 1;
    int all = 1;
    for (int32_t v = 0; v < n && all; ++v) all = (RC[v] == 0);
    if (all) { s.converged = 1; break; }
  }
  int32_t a = 0;
  for (int32_t v = 0; v < n; ++v) a += VA[v];
  s.affected = a;
  free(VA); free(RC); free(C);
  if (st) *st = s;
  return ORC_OK;
}

/* ----------------------------------------------------------------------- */
/* Sampled rows straight from raw edges (for checks at large sizes)         */
/* ----------------------------------------------------------------------- */

/*
 * For each of the k vertices in `which`, computes its row of the graph
 * G^1 = apply(build(raw edges, self_loops), batch): its out-row (dir = 0,
 * targets) or in-row (dir = 1, sources), sorted and unique. One scan of the
 * raw edges per call; no full graph is formed. Rows are written to
 * row_idx[row_off[i] .. row_off[i + 1]) and row_off has k + 1 entries; the
 * caller sizes row_idx with cap entries; returns the number written, or
 * ORC_ENOMEM when cap is too small or memory runs out.
 * n_batch_del / n_batch_ins == 0 gives the rows of G^0.
 */
int64_t orc_sample_rows(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                        int self_loops, int64_t n_del, const int32_t* del_src,
                        const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                        const int32_t* ins_dst, int dir, int32_t k, const int32_t* which,
                        int64_t* row_off, int32_t* row_idx, int64_t cap) {
  if (n <= 0 || k < 0) return ORC_EINVAL;
  /* slot[v] = index of v in `which` + 1, or 0 */
  int32_t* slot = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int64_t* cnt = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  if (!slot || !cnt) { free(slot); free(cnt); return ORC_ENOMEM; }
  for (int32_t i = 0; i < k; ++i) slot[which[i]] = i + 1;
  /* gather candidate (row owner, neighbour) keys */
  int64_t nk = 0, kcap = 1024;
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)kcap);
  if (!keys) { free(slot); free(cnt); return ORC_ENOMEM; }
#define PUSH_KEY(a, b)                                                                  \
  do {                                                                                  \
    if (nk == kcap) {                                                                   \
      kcap *= 2;                                                                        \
      uint64_t* t_ = (uint64_t*)realloc(keys, sizeof(uint64_t) * (size_t)kcap);        \
      if (!t_) { free(keys); free(slot); free(cnt); return ORC_ENOMEM; }                \
      keys = t_;                                                                        \
    }                                                                                   \
    keys[nk++] = key_of((a), (b));                                                      \
  } while (0)
  for (int64_t i = 0; i < m_raw; ++i) {
    int32_t owner = dir == 0 ? src[i] : dst[i];
    int32_t other = dir == 0 ? dst[i] : src[i];
    if (slot[owner]) PUSH_KEY(owner, other);
  }
  if (self_loops)
    for (int32_t i = 0; i < k; ++i) PUSH_KEY(which[i], which[i]);
  nk = sort_unique(keys, nk);
  /* batch: real deletions / insertions restricted to the sampled rows */
  uint64_t* dk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_del > 0 ? n_del : 1));
  uint64_t* ik = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_ins > 0 ? n_ins : 1));
  if (!dk || !ik) { free(dk); free(ik); free(keys); free(slot); free(cnt); return ORC_ENOMEM; }
  int64_t nd = 0, ni = 0;
  for (int64_t i = 0; i < n_ins; ++i) {
    int32_t owner = dir == 0 ? ins_src[i] : ins_dst[i];
    int32_t other = dir == 0 ? ins_dst[i] : ins_src[i];
    if (slot[owner]) ik[ni++] = key_of(owner, other);
  }
  ni = sort_unique(ik, ni);
  for (int64_t i = 0; i < n_del; ++i) {
    int32_t owner = dir == 0 ? del_src[i] : del_dst[i];
    int32_t other = dir == 0 ? del_dst[i] : del_src[i];
    if (!slot[owner]) continue;
    if (self_loops && owner == other) continue;
    uint64_t x = key_of(owner, other);
    if (has_key(ik, ni, x)) continue;           /* re-inserted: stays */
    dk[nd++] = x;
  }
  nd = sort_unique(dk, nd);
  /* merge: old keys minus deletions, plus insertions */
  uint64_t* all = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nk + ni + 1));
  if (!all) { free(dk); free(ik); free(keys); free(slot); free(cnt); return ORC_ENOMEM; }
  int64_t na = 0;
  for (int64_t i = 0; i < nk; ++i)
    if (!has_key(dk, nd, keys[i])) all[na++] = keys[i];
  for (int64_t i = 0; i < ni; ++i) all[na++] = ik[i];
  na = sort_unique(all, na);
  int64_t rc = na;
  if (na > cap) rc = ORC_ENOMEM;
  else {
    for (int64_t i = 0; i < na; ++i) cnt[slot[key_hi(all[i])]]++;
    /* rows in the order of `which` */
    row_off[0] = 0;
    for (int32_t i = 0; i < k; ++i) row_off[i + 1] = row_off[i] + cnt[i + 1];
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k + 1));
    if (!pos) rc = ORC_ENOMEM;
    else {
      for (int32_t i = 0; i < k; ++i) pos[i] = row_off[i];
      for (int64_t i = 0; i < na; ++i) {
        int32_t s = slot[key_hi(all[i])] - 1;
        row_idx[pos[s]++] = key_lo(all[i]);
      }
      free(pos);
    }
  }
#undef PUSH_KEY
  free(all); free(dk); free(ik); free(keys); free(slot); free(cnt);
  return rc;
}
