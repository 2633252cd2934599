/*
 * Seeded synthetic workload generators for dynamic PageRank experiments.
 *
 * These produce raw edge lists and edge-update batches shaped like the
 * paper's workloads (Sec. 5.1.3 datasets, Sec. 5.1.4 batch generation):
 * R-MAT graphs stand in for the web/social graphs of Table 2, a 2D grid with
 * a few long-range arcs stands in for the road networks, and batches are
 * uniform random insertions of vertex pairs plus uniform deletions of edges.
 *
 * This file holds no PageRank arithmetic and no graph construction: it only
 * draws random numbers. Both the CPU oracle's tests and the GPU path's tests
 * and benchmark take their inputs from here.
 *
 * Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-style: draw k of
 * stream s is mix64(key(s) + (k + 1) * 0x9E3779B97F4A7C15). Each edge owns a
 * fixed range of counters, so the output does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Stream key for (seed, stream id). */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * GOLDEN + mix64(stream + 0x1234567ULL));
}

static inline uint64_t draw(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * GOLDEN);
}

/* Uniform integer in [0, bound) from one 64-bit draw (Lemire's multiply-shift;
 * the bias is below 2^-32 for bound < 2^32). */
static inline uint64_t below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

int gen_version(void) { return 1; }

/* ----------------------------------------------------------------------- */
/* Thread fan-out helper                                                    */
/* ----------------------------------------------------------------------- */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;

static void* range_trampoline(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(int64_t count, int threads, range_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  if (count < 65536 || threads == 1) { fn(ctx, 0, count); return; }
  pthread_t tid[64];
  range_job jobs[64];
  int64_t per = (count + threads - 1) / threads;
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    int64_t lo = (int64_t)t * per, hi = lo + per;
    if (lo >= count) break;
    if (hi > count) hi = count;
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
    if (pthread_create(&tid[t], NULL, range_trampoline, &jobs[t]) != 0) {
      fn(ctx, lo, hi);              /* run inline if a thread cannot start */
      jobs[t].fn = NULL;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (jobs[t].fn) pthread_join(tid[t], NULL);
}

/* ----------------------------------------------------------------------- */
/* R-MAT                                                                    */
/* ----------------------------------------------------------------------- */

typedef struct {
  int scale;
  uint32_t t_a, t_ab, t_abc;     /* 16-bit quadrant thresholds */
  uint64_t key;
  const int32_t* perm;           /* label permutation of [0, 2^scale) */
  int32_t* src;
  int32_t* dst;
} rmat_ctx;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
  rmat_ctx* c = (rmat_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t row = 0, col = 0, r = 0;
    for (int lvl = 0; lvl < c->scale; ++lvl) {
      if ((lvl & 3) == 0) r = draw(c->key, (uint64_t)i * 8 + (uint64_t)(lvl >> 2));
      uint32_t u = (uint32_t)(r & 0xFFFF);
      r >>= 16;
      row <<= 1; col <<= 1;
      if (u < c->t_a) {
      } else if (u < c->t_ab) {
        col |= 1;
      } else if (u < c->t_abc) {
        row |= 1;
      } else {
        row |= 1; col |= 1;
      }
    }
    c->src[i] = c->perm ? c->perm[row] : (int32_t)row;
    c->dst[i] = c->perm ? c->perm[col] : (int32_t)col;
  }
}

/*
 * R-MAT edge draws (Chakrabarti, Zhan, Faloutsos 2004) at 2^scale labels.
 * Each of the m draws descends `scale` levels, choosing quadrant a/b/c/d with
 * the given probabilities (quantised to 1/65536). Labels are then permuted by
 * a seeded Fisher-Yates shuffle (as Graph500 does), so vertex ids carry no
 * locality. Duplicates and self-loops are kept: the caller's graph builder
 * removes or adds them. scale <= 31, m >= 0.
 */
int gen_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
             int permute, int threads, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 31 || m < 0 || !src || !dst) return -1;
  rmat_ctx ctx;
  ctx.scale = scale;
  ctx.t_a = (uint32_t)llround(a * 65536.0);
  ctx.t_ab = (uint32_t)llround((a + b) * 65536.0);
  ctx.t_abc = (uint32_t)llround((a + b + c) * 65536.0);
  ctx.key = stream_key(seed, 1);
  ctx.src = src; ctx.dst = dst; ctx.perm = NULL;
  int32_t* perm = NULL;
  if (permute) {
    int64_t nl = (int64_t)1 << scale;
    perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)nl);
    if (!perm) return -2;
    for (int64_t i = 0; i < nl; ++i) perm[i] = (int32_t)i;
    uint64_t pk = stream_key(seed, 2);
    for (int64_t i = nl - 1; i > 0; --i) {
      int64_t j = (int64_t)below(draw(pk, (uint64_t)i), (uint64_t)(i + 1));
      int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    ctx.perm = perm;
  }
  parallel_for(m, threads, rmat_range, &ctx);
  free(perm);
  return 0;
}

/* Keeps only draws whose endpoints are both < n (for n not a power of two).
 * Compacts in place and returns the number kept. */
int64_t gen_filter_below(int64_t m, int32_t n, int32_t* src, int32_t* dst) {
  int64_t k = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (src[i] < n && dst[i] < n) { src[k] = src[i]; dst[k] = dst[i]; ++k; }
  }
  return k;
}

/* ----------------------------------------------------------------------- */
/* 2D grid with long-range arcs (road-network stand-in)                     */
/* ----------------------------------------------------------------------- */

/* Number of arcs gen_grid writes: 4 L (L - 1) grid arcs plus `shortcuts`. */
int64_t gen_grid_count(int32_t L, int64_t shortcuts) {
  return 4LL * L * (L - 1) + shortcuts;
}

/*
 * L x L grid, vertex (r, c) has id r * L + c. Every grid neighbour pair is
 * joined in both directions. Then `shortcuts` uniform random arcs u -> v with
 * u != v are appended. Output order: for each vertex in id order, its arcs to
 * up, down, left, right neighbours that exist; then the shortcuts.
 */
int gen_grid(int32_t L, int64_t shortcuts, uint64_t seed, int32_t* src, int32_t* dst) {
  if (L < 2 || shortcuts < 0 || (int64_t)L * L > 0x7FFFFFFF) return -1;
  int64_t k = 0;
  for (int32_t r = 0; r < L; ++r) {
    for (int32_t c = 0; c < L; ++c) {
      int32_t v = r * L + c;
      if (r > 0)     { src[k] = v; dst[k] = v - L; ++k; }
      if (r < L - 1) { src[k] = v; dst[k] = v + L; ++k; }
      if (c > 0)     { src[k] = v; dst[k] = v - 1; ++k; }
      if (c < L - 1) { src[k] = v; dst[k] = v + 1; ++k; }
    }
  }
  uint64_t key = stream_key(seed, 3);
  int64_t n = (int64_t)L * L;
  for (int64_t i = 0; i < shortcuts; ++i) {
    uint64_t ctr = (uint64_t)i * 16;
    int64_t u = (int64_t)below(draw(key, ctr), (uint64_t)n);
    int64_t v = (int64_t)below(draw(key, ctr + 1), (uint64_t)n);
    for (uint64_t t = 2; v == u && t < 16; ++t) v = (int64_t)below(draw(key, ctr + t), (uint64_t)n);
    if (v == u) v = (u + 1) % n;
    src[k] = (int32_t)u; dst[k] = (int32_t)v; ++k;
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Batches                                                                  */
/* ----------------------------------------------------------------------- */

typedef struct {
  int32_t n;
  uint64_t key_ins, key_del;
  const int32_t* pool_src;
  const int32_t* pool_dst;
  int64_t pool_m;
  int32_t *ins_src, *ins_dst, *del_src, *del_dst;
  int64_t n_ins, n_del;
} batch_ctx;

static void batch_ins_range(void* p, int64_t lo, int64_t hi) {
  batch_ctx* c = (batch_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t ctr = (uint64_t)i * 16;
    int32_t u = (int32_t)below(draw(c->key_ins, ctr), (uint64_t)c->n);
    int32_t v = (int32_t)below(draw(c->key_ins, ctr + 1), (uint64_t)c->n);
    for (uint64_t t = 2; v == u && t < 16; ++t)
      v = (int32_t)below(draw(c->key_ins, ctr + t), (uint64_t)c->n);
    if (v == u) v = (int32_t)((u + 1) % c->n);
    c->ins_src[i] = u; c->ins_dst[i] = v;
  }
}

static void batch_del_range(void* p, int64_t lo, int64_t hi) {
  batch_ctx* c = (batch_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t ctr = (uint64_t)i * 64;
    int64_t j = (int64_t)below(draw(c->key_del, ctr), (uint64_t)c->pool_m);
    for (uint64_t t = 1; c->pool_src[j] == c->pool_dst[j] && t < 64; ++t)
      j = (int64_t)below(draw(c->key_del, ctr + t), (uint64_t)c->pool_m);
    c->del_src[i] = c->pool_src[j]; c->del_dst[i] = c->pool_dst[j];
  }
}

/*
 * Random batch (Sec. 5.1.4): n_ins insertions of uniform vertex pairs u != v
 * and n_del deletions drawn uniformly (with replacement) from the given edge
 * pool, skipping pool entries that are self-loops. Whether an insertion hits
 * an existing edge or a deletion repeats is left to the graph update, which
 * treats both as no-ops. Needs n >= 2 and a pool with a non-loop edge when
 * n_del > 0.
 */
int gen_batch_uniform(int32_t n, int64_t n_ins, int64_t n_del, uint64_t seed,
                      const int32_t* pool_src, const int32_t* pool_dst, int64_t pool_m,
                      int threads, int32_t* ins_src, int32_t* ins_dst,
                      int32_t* del_src, int32_t* del_dst) {
  if (n < 2 || n_ins < 0 || n_del < 0) return -1;
  if (n_del > 0 && (pool_m <= 0 || !pool_src || !pool_dst)) return -1;
  batch_ctx c;
  memset(&c, 0, sizeof c);
  c.n = n;
  c.key_ins = stream_key(seed, 10);
  c.key_del = stream_key(seed, 11);
  c.pool_src = pool_src; c.pool_dst = pool_dst; c.pool_m = pool_m;
  c.ins_src = ins_src; c.ins_dst = ins_dst; c.del_src = del_src; c.del_dst = del_dst;
  c.n_ins = n_ins; c.n_del = n_del;
  parallel_for(n_ins, threads, batch_ins_range, &c);
  parallel_for(n_del, threads, batch_del_range, &c);
  return 0;
}

/*
 * Localised batch on an L x L grid: all endpoints fall inside one random
 * square window of side w = min(L, ceil(4 sqrt(b))) cells, b = n_ins + n_del.
 * Deletions pick a random cell of the window and a random direction whose
 * neighbour is also inside; insertions pick two distinct cells of the window.
 * Writes the window origin to origin[0..1] (row, col) when origin != NULL.
 */
int gen_batch_grid_local(int32_t L, int64_t n_ins, int64_t n_del, uint64_t seed,
                         int32_t* ins_src, int32_t* ins_dst, int32_t* del_src,
                         int32_t* del_dst, int32_t* origin) {
  if (L < 2 || n_ins < 0 || n_del < 0) return -1;
  int64_t b = n_ins + n_del;
  int64_t w = (int64_t)ceil(4.0 * sqrt((double)(b > 0 ? b : 1)));
  if (w < 2) w = 2;
  if (w > L) w = L;
  uint64_t key = stream_key(seed, 20);
  int64_t r0 = (int64_t)below(draw(key, 0), (uint64_t)(L - w + 1));
  int64_t c0 = (int64_t)below(draw(key, 1), (uint64_t)(L - w + 1));
  if (origin) { origin[0] = (int32_t)r0; origin[1] = (int32_t)c0; }
  uint64_t ki = stream_key(seed, 21), kd = stream_key(seed, 22);
  int64_t cells = w * w;
  for (int64_t i = 0; i < n_ins; ++i) {
    uint64_t ctr = (uint64_t)i * 16;
    int64_t a = (int64_t)below(draw(ki, ctr), (uint64_t)cells);
    int64_t z = (int64_t)below(draw(ki, ctr + 1), (uint64_t)cells);
    for (uint64_t t = 2; z == a && t < 16; ++t) z = (int64_t)below(draw(ki, ctr + t), (uint64_t)cells);
    if (z == a) z = (a + 1) % cells;
    ins_src[i] = (int32_t)((r0 + a / w) * L + c0 + a % w);
    ins_dst[i] = (int32_t)((r0 + z / w) * L + c0 + z % w);
  }
  static const int dr[4] = {-1, 1, 0, 0}, dc[4] = {0, 0, -1, 1};
  for (int64_t i = 0; i < n_del; ++i) {
    uint64_t ctr = (uint64_t)i * 64;
    for (uint64_t t = 0;; t += 2) {
      int64_t a = (int64_t)below(draw(kd, ctr + t), (uint64_t)cells);
      int d = (int)below(draw(kd, ctr + t + 1), 4);
      int64_t r = a / w, c = a % w, r2 = r + dr[d], c2 = c + dc[d];
      if ((r2 >= 0 && r2 < w && c2 >= 0 && c2 < w) || t >= 62) {
        if (!(r2 >= 0 && r2 < w && c2 >= 0 && c2 < w)) { r2 = r; c2 = (c + 1 < w) ? c + 1 : c - 1; }
        del_src[i] = (int32_t)((r0 + r) * L + c0 + c);
        del_dst[i] = (int32_t)((r0 + r2) * L + c0 + c2);
        break;
      }
    }
  }
  return 0;
}

/* Uniform doubles in [0, 1) (53-bit), for drawing graph sizes and degrees. */
void gen_uniform(uint64_t seed, uint64_t stream, int64_t count, double* out) {
  uint64_t key = stream_key(seed, 100 + stream);
  for (int64_t i = 0; i < count; ++i)
    out[i] = (double)(draw(key, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
}
