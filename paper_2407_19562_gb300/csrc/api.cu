// C ABI of libdfpr (declared in include/dfpr.h): argument checks, device and
// stream handling, host <-> device staging and status codes. Every entry
// point catches the library's internal failures and returns a status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "common.cuh"
#include "df.cuh"
#include "graph.cuh"
#include "primitives.cuh"

namespace dfpr {

namespace {
thread_local std::string t_err;
std::mutex g_alloc_mu;
dfpr_alloc_fn g_alloc = nullptr;
dfpr_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
}  // namespace

std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { t_err = msg; }
const char* get_error() { return t_err.c_str(); }

void* dev_alloc(size_t bytes, cudaStream_t s, FreeRec* rec) {
  dfpr_alloc_fn fa;
  FreeRec r;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    fa = g_alloc;
    r.fn = g_free;
    r.ctx = g_alloc_ctx;
  }
  void* p = nullptr;
  if (fa) {
    p = fa(bytes, (void*)s, r.ctx);
  } else {
    r.fn = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) {
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
    throw Fail{DFPR_ENOMEM};
  }
  *rec = r;
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s, const FreeRec& rec) {
  if (!p) return;
  if (rec.fn) rec.fn(p, bytes, (void*)s, rec.ctx);
  else cudaFree(p);
}

namespace {

constexpr int kNT = 256;

#define GRID_STRIDE(i, n)                                                             \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
       i += (long long)gridDim.x * blockDim.x)

// out[u] = in[perm[u]] (caller order from internal order; perm may be null).
template <class T>
__global__ void k_ranks_out(const T* __restrict__ in, const int32_t* __restrict__ perm,
                            double* __restrict__ out, long long n) {
  GRID_STRIDE(u, n) out[u] = (double)in[perm ? perm[u] : u];
}
// out[perm[u]] = in[u] (internal order from caller order).
template <class T>
__global__ void k_ranks_in(const double* __restrict__ in, const int32_t* __restrict__ perm,
                           T* __restrict__ out, long long n) {
  GRID_STRIDE(u, n) out[perm ? perm[u] : u] = (T)in[u];
}

// Makes the graph's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) DFPR_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// One call at a time per graph.
struct BusyGuard {
  dfpr_graph* g;
  explicit BusyGuard(dfpr_graph* gr) : g(gr) {
    int z = 0;
    if (!g->busy.compare_exchange_strong(z, 1)) {
      g = nullptr;
      set_error("another call on this graph is in progress");
      throw Fail{DFPR_EBUSY};
    }
  }
  ~BusyGuard() {
    if (g) g->busy.store(0);
  }
};

// Device copy of a caller array (or the caller's device pointer itself).
template <class T>
const T* stage_in(dfpr_graph* g, DevArray<T>& tmp, const T* p, long long n, int on_device) {
  if (n <= 0) return nullptr;
  if (on_device) return p;
  tmp.reset((size_t)n, g->stream);
  DFPR_CUDA(cudaMemcpyAsync(tmp.p, p, sizeof(T) * n, cudaMemcpyHostToDevice, g->stream));
  return tmp.p;
}

void check_params(const dfpr_params& p) {
  DFPR_REQUIRE(p.alpha > 0.0 && p.alpha < 1.0, DFPR_EINVAL, "alpha must lie in (0, 1)");
  DFPR_REQUIRE(p.tol > 0.0 && std::isfinite(p.tol), DFPR_EINVAL, "tol must be positive");
  DFPR_REQUIRE(p.max_iter >= 1, DFPR_EINVAL, "max_iter must be >= 1");
  DFPR_REQUIRE(p.mode >= DFPR_MODE_WORKLIST && p.mode <= DFPR_MODE_JACOBI, DFPR_EINVAL,
               "unknown mode");
  DFPR_REQUIRE(p.grid_ctas >= 0, DFPR_EINVAL, "grid_ctas must be >= 0");
  DFPR_REQUIRE(p.fault_delay_prob >= 0.0 && p.fault_delay_prob <= 1.0, DFPR_EINVAL,
               "fault_delay_prob must lie in [0, 1]");
  DFPR_REQUIRE(p.fault_delay_us >= 0.0 && p.fault_delay_us <= 1e6, DFPR_EINVAL,
               "fault_delay_us must lie in [0, 1e6]");
  DFPR_REQUIRE(p.fault_crash_warps >= 0, DFPR_EINVAL, "fault_crash_warps must be >= 0");
  DFPR_REQUIRE(p.gather_split == 0 || (p.gather_split >= 256 && p.gather_split <= (1 << 24)),
               DFPR_EINVAL, "gather_split must be 0 or lie in [256, 2^24]");
  DFPR_REQUIRE(p.mark_split == 0 || (p.mark_split >= 256 && p.mark_split <= (1 << 24)),
               DFPR_EINVAL, "mark_split must be 0 or lie in [256, 2^24]");
  DFPR_REQUIRE(p.helping == 0 || p.helping == 1, DFPR_EINVAL, "helping must be 0 or 1");
  DFPR_REQUIRE(!(p.fault_crash_warps > 0 && p.mode == DFPR_MODE_JACOBI), DFPR_EINVAL,
               "crash-stop faults need a lock-free schedule: the jacobi schedule's iteration "
               "barrier would never complete (Sec. 5.4)");
}


}  // namespace

dfpr_status run_update(dfpr_graph* g, const dfpr_params* pp, dfpr_stats* st, RunKind kind) {
  dfpr_params p;
  if (pp) p = *pp;
  else dfpr_default_params(&p);
  check_params(p);
  DFPR_REQUIRE(g->max_degree <= kDegreeLimit, DFPR_EINVAL,
               "a vertex has more than 2^25 - 1 in- or out-edges, the update kernels' limit");
  DFPR_REQUIRE(!(p.normalize && g->nparts > 1), DFPR_EINVAL,
               "normalize is not supported for a set of graphs");
  if (g->cfg.dead_end == DFPR_TELEPORT)
    DFPR_REQUIRE(p.mode == DFPR_MODE_JACOBI, DFPR_EINVAL,
                 "teleport dead-end handling is supported by the jacobi schedule only");
  {
    // a launch's gather (and mark) tokens must fit half the token ring each
    const long long min_split = std::max<long long>(256, (g->m + (1ll << 20) - 1) >> 20);
    DFPR_REQUIRE(p.gather_split == 0 || p.gather_split >= min_split, DFPR_EINVAL,
                 "gather_split must be at least max(256, edges / 2^20)");
    DFPR_REQUIRE(p.mark_split == 0 || p.mark_split >= min_split, DFPR_EINVAL,
                 "mark_split must be at least max(256, edges / 2^20)");
  }
  dfpr_stats local;
  memset(&local, 0, sizeof local);
  local.rank_sum = NAN;
  if (kind == kRunDF && g->pend.n_src == 0 && g->pend.n_dst == 0) {
    if (st) *st = local;
    return DFPR_OK;
  }
  dfpr_status r = run_iteration(g, p, kind, &local);
  g->d_before_valid = false;  // the ranks were recomputed
  if (p.normalize && r == DFPR_OK) local.rank_sum = rank_sum(g);
  if (st) *st = local;
  if (r != DFPR_OK)
    set_error(r == DFPR_ETIMEOUT ? "the time budget ran out before convergence"
                                 : "the iteration cap was reached before convergence");
  return r;
}

}  // namespace dfpr

using namespace dfpr;

#define API_BEGIN try {
#define API_END                                              \
  }                                                          \
  catch (const Fail& f) {                                    \
    return f.st;                                             \
  }                                                          \
  catch (const std::bad_alloc&) {                            \
    set_error("host allocation failed");                     \
    return DFPR_ENOMEM;                                      \
  }                                                          \
  catch (...) {                                              \
    set_error("unexpected internal error");                  \
    return DFPR_ECUDA;                                       \
  }

extern "C" {

void dfpr_default_config(dfpr_graph_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->precision = DFPR_FP64;
  cfg->dead_end = DFPR_SELF_LOOPS;
  cfg->row_slack = 0.125;
  cfg->min_slack = 2;
  cfg->reorder = 1;
  cfg->tail_slack = 0.125;
}

void dfpr_default_params(dfpr_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->alpha = 0.85;
  p->tol = 1e-10;
  p->frontier_tol = 0.0;
  p->max_iter = 500;
  p->mode = DFPR_MODE_WORKLIST;
  p->helping = 1;
  p->normalize = 0;
  p->grid_ctas = 0;
  p->timeout_ms = 60000.0;
  p->fault_delay_prob = 0.0;
  p->fault_delay_us = 0.0;
  p->fault_crash_warps = 0;
  p->fault_seed = 0u;
  p->gather_split = 0;
  p->mark_split = 0;
}

int32_t dfpr_version(void) { return 100; }

int64_t dfpr_kernel_launches(void) { return (int64_t)g_launches.load(); }

const char* dfpr_last_error(void) { return get_error(); }

dfpr_status dfpr_set_allocator(dfpr_alloc_fn alloc, dfpr_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    set_error("dfpr_set_allocator: give both functions or neither");
    return DFPR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return DFPR_OK;
}

static dfpr_status load_impl(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                             int on_device, void* cuda_stream, const dfpr_graph_config* cfg,
                             int32_t k, const int32_t* vertex_offsets, dfpr_graph** out) {
  set_error("");
  if (!out) {
    set_error("dfpr_graph_load: out is NULL");
    return DFPR_EINVAL;
  }
  *out = nullptr;
  if (n <= 0 || m < 0 || (m > 0 && (!src || !dst))) {
    set_error("dfpr_graph_load: need n > 0, m >= 0 and edge arrays when m > 0");
    return DFPR_EINVAL;
  }
  dfpr_graph_config c;
  if (cfg) c = *cfg;
  else dfpr_default_config(&c);
  if ((c.precision != DFPR_FP64 && c.precision != DFPR_FP32) ||
      (c.dead_end != DFPR_SELF_LOOPS && c.dead_end != DFPR_TELEPORT) || c.row_slack < 0 ||
      c.min_slack < 0 || c.tail_slack < 0) {
    set_error("dfpr_graph_load: invalid config");
    return DFPR_EINVAL;
  }
  if (m + (c.dead_end == DFPR_SELF_LOOPS ? (long long)n : 0ll) > kEdgeLimit) {
    set_error("dfpr_graph_load: a graph holds at most 2^32 - 2 edges, self-loops included");
    return DFPR_EINVAL;
  }
  if (k > 1 && c.dead_end == DFPR_TELEPORT) {
    set_error("dfpr_graph_load_parts: teleport dead-end handling is not supported for a set");
    return DFPR_EINVAL;
  }
  dfpr_graph* g = nullptr;
  API_BEGIN
  g = new dfpr_graph();
  g->cfg = c;
  g->n = n;
  g->bits = id_bits(n);
  DFPR_CUDA(cudaGetDevice(&g->device));
  DFPR_CUDA(cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device));
  if (cuda_stream) {
    g->stream = (cudaStream_t)cuda_stream;
  } else {
    DFPR_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->own_stream = true;
  }
  DFPR_CUDA(cudaMallocHost(&g->pinned, 16 * sizeof(unsigned long long)));
  g->host_sync.reset(16, g->stream);
  DFPR_CUDA(cudaMemsetAsync(g->host_sync.p, 0, 16 * sizeof(unsigned long long), g->stream));
  if (k > 1) {
    g->nparts = k;
    g->part_off_host.assign(vertex_offsets, vertex_offsets + k + 1);
    g->part_off.reset((size_t)k + 1, g->stream);
    DFPR_CUDA(cudaMemcpyAsync(g->part_off.p, g->part_off_host.data(), sizeof(int32_t) * (k + 1),
                              cudaMemcpyHostToDevice, g->stream));
    g->part_done.reset((size_t)k, g->stream);
    DFPR_CUDA(cudaMemsetAsync(g->part_done.p, 0, sizeof(unsigned long long) * k, g->stream));
    g->part_ms.assign((size_t)k, 0.0);
  }
  {
    DevArray<int32_t> ts, td;
    const int32_t* ds = stage_in(g, ts, src, m, on_device);
    const int32_t* dd = stage_in(g, td, dst, m, on_device);
    graph_build(g, ds, dd, m);
    DFPR_CUDA(cudaStreamSynchronize(g->stream));
  }
  alloc_iteration_state(g);
  reset_ranks(g);
  DFPR_CUDA(cudaStreamSynchronize(g->stream));
  *out = g;
  return DFPR_OK;
  }
  catch (const Fail& f) {
    if (g) dfpr_graph_free(g);
    return f.st;
  }
  catch (const std::bad_alloc&) {
    if (g) dfpr_graph_free(g);
    set_error("host allocation failed");
    return DFPR_ENOMEM;
  }
  catch (...) {
    if (g) dfpr_graph_free(g);
    set_error("unexpected internal error");
    return DFPR_ECUDA;
  }
}

dfpr_status dfpr_graph_load(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            int on_device, void* cuda_stream, const dfpr_graph_config* cfg,
                            dfpr_graph** out) {
  return load_impl(n, m, src, dst, on_device, cuda_stream, cfg, 1, nullptr, out);
}

dfpr_status dfpr_graph_load_parts(int32_t k, const int32_t* vertex_offsets, int64_t m,
                                  const int32_t* src, const int32_t* dst, int on_device,
                                  void* cuda_stream, const dfpr_graph_config* cfg,
                                  dfpr_graph** out) {
  if (out) *out = nullptr;
  if (k < 1 || !vertex_offsets || vertex_offsets[0] != 0) {
    set_error("dfpr_graph_load_parts: need k >= 1 and vertex_offsets[0] == 0");
    return DFPR_EINVAL;
  }
  for (int32_t i = 0; i < k; ++i)
    if (vertex_offsets[i + 1] <= vertex_offsets[i]) {
      set_error("dfpr_graph_load_parts: every graph needs at least one vertex (offsets must increase)");
      return DFPR_EINVAL;
    }
  return load_impl(vertex_offsets[k], m, src, dst, on_device, cuda_stream, cfg, k, vertex_offsets, out);
}

dfpr_status dfpr_graph_parts(const dfpr_graph* g, int32_t* k) {
  if (!g || !k) {
    set_error("dfpr_graph_parts: NULL argument");
    return DFPR_EINVAL;
  }
  *k = g->nparts;
  return DFPR_OK;
}

dfpr_status dfpr_get_part_times(const dfpr_graph* g, double* ms) {
  if (!g || !ms) {
    set_error("dfpr_get_part_times: NULL argument");
    return DFPR_EINVAL;
  }
  for (int i = 0; i < g->nparts; ++i) ms[i] = i < (int)g->part_ms.size() ? g->part_ms[i] : 0.0;
  return DFPR_OK;
}

dfpr_status dfpr_graph_free(dfpr_graph* g) {
  if (!g) return DFPR_OK;
  int idle = 0;
  if (!g->busy.compare_exchange_strong(idle, 1)) {
    set_error("dfpr_graph_free: another call on this graph is in progress");
    return DFPR_EBUSY;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  cudaStream_t s = g->stream;
  const bool own = g->own_stream;
  unsigned long long* pinned = g->pinned;
  std::vector<cudaStream_t> retired;
  retired.swap(g->retired_streams);
  if (g->cap_exec) cudaGraphExecDestroy(g->cap_exec);
  for (cudaEvent_t e : g->cap_ev)
    if (e) cudaEventDestroy(e);
  if (g->cap_host) cudaFreeHost(g->cap_host);
  // device arrays are released by their destructors, with the streams they
  // were allocated on still alive (an installed allocator may use them)
  delete g;
  if (pinned) cudaFreeHost(pinned);
  if (own && s) cudaStreamDestroy(s);
  for (cudaStream_t r : retired) cudaStreamDestroy(r);
  if (prev >= 0) cudaSetDevice(prev);
  return DFPR_OK;
}

dfpr_status dfpr_graph_set_stream(dfpr_graph* g, void* cuda_stream) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  DFPR_CUDA(cudaStreamSynchronize(g->stream));
  if (g->own_stream) {
    // kept until the graph is freed: arrays allocated on it record it
    g->retired_streams.push_back(g->stream);
    g->own_stream = false;
  }
  if (cuda_stream) {
    g->stream = (cudaStream_t)cuda_stream;
  } else {
    DFPR_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->own_stream = true;
  }
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_graph_set_capture(dfpr_graph* g, int32_t enable) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  g->capture = enable != 0;
  if (!g->capture && g->cap_exec) {
    DFPR_CUDA(cudaStreamSynchronize(g->stream));
    DFPR_CUDA(cudaGraphExecDestroy(g->cap_exec));
    g->cap_exec = nullptr;
    g->cap_key.clear();
  }
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_graph_capture_info(const dfpr_graph* g, int64_t* captures, int64_t* replays) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  if (captures) *captures = g->cap_captures;
  if (replays) *replays = g->cap_replays;
  return DFPR_OK;
}

dfpr_status dfpr_graph_info(const dfpr_graph* g, int32_t* n, int64_t* m, int32_t* device) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (device) *device = g->device;
  return DFPR_OK;
}

dfpr_status dfpr_apply_batch(dfpr_graph* g, int64_t n_del, const int32_t* del_src,
                             const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                             const int32_t* ins_dst, int on_device, int64_t* n_applied) {
  if (n_applied) n_applied[0] = n_applied[1] = 0;
  if (!g || n_del < 0 || n_ins < 0 || (n_del > 0 && (!del_src || !del_dst)) ||
      (n_ins > 0 && (!ins_src || !ins_dst))) {
    set_error("dfpr_apply_batch: invalid arguments");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DFPR_REQUIRE(n_del + n_ins <= kEdgeLimit && g->m + n_ins <= kEdgeLimit, DFPR_EINVAL,
               "dfpr_apply_batch: a batch, and a graph after it, hold at most 2^32 - 2 edges");
  DeviceGuard dg(g->device);
  DevArray<int32_t> a, b, c, d;
  const int32_t* ds = stage_in(g, a, del_src, n_del, on_device);
  const int32_t* dd = stage_in(g, b, del_dst, n_del, on_device);
  const int32_t* is = stage_in(g, c, ins_src, n_ins, on_device);
  const int32_t* id = stage_in(g, d, ins_dst, n_ins, on_device);
  long long applied[2] = {0, 0};
  if (g->cfg.dead_end == DFPR_TELEPORT && !g->d_before_valid) {
    g->d_before = dangling_mass(g);  // the D the current ranks were computed with
    g->d_before_valid = true;
  }
  graph_apply(g, ds, dd, n_del, is, id, n_ins, applied);
  DFPR_CUDA(cudaStreamSynchronize(g->stream));
  if (n_applied) {
    n_applied[0] = applied[0];
    n_applied[1] = applied[1];
  }
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_df_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  return run_update(g, p, stats, kRunDF);
  API_END
}

namespace {

// Runs the pending update once per plan (mode, grid_ctas, gather_split,
// mark_split), each time from the same ranks, contributions and pending
// change set, timing the whole call with CUDA events; then restores that
// state once more and runs the fastest plan, which stays applied.
dfpr_status autotune_plans(dfpr_graph* g, dfpr_params* p, int32_t k, const int32_t* plans,
                           double* trial_ms, dfpr_stats* stats) {
  DFPR_REQUIRE(g->pend.n_src > 0 || g->pend.n_dst > 0, DFPR_EINVAL,
               "dfpr_autotune: no pending changes to time the candidates on");
  auto plan_params = [&](int32_t i) {
    dfpr_params q = *p;
    q.mode = plans[4 * i];
    q.grid_ctas = plans[4 * i + 1];
    q.gather_split = plans[4 * i + 2];
    q.mark_split = plans[4 * i + 3];
    return q;
  };
  for (int32_t i = 0; i < k; ++i) {
    const dfpr_params q = plan_params(i);
    check_params(q);
    if (g->cfg.dead_end == DFPR_TELEPORT)
      DFPR_REQUIRE(q.mode == DFPR_MODE_JACOBI, DFPR_EINVAL,
                   "dfpr_autotune: teleport graphs run the jacobi schedule only");
  }
  cudaStream_t s = g->stream;
  const long long n_src = g->pend.n_src, n_dst = g->pend.n_dst;
  const bool fp64 = g->cfg.precision == DFPR_FP64;
  const size_t r_bytes = (fp64 ? sizeof(double) : sizeof(float)) * (size_t)g->n;
  const size_t c_bytes = (fp64 ? sizeof(long long) : sizeof(float)) * (size_t)g->n;
  // the jacobi schedule swaps its two vectors: look the current ones up each time
  auto vectors = [&](void** R, void** C) {
    *R = fp64 ? (void*)g->R64.p : (void*)g->R32.p;
    *C = fp64 ? (void*)g->C64.p : (void*)g->C32.p;
  };
  DevArray<unsigned char> snap;  // the ranks and contributions every trial starts from
  snap.reset(r_bytes + c_bytes, s);
  void *R, *C;
  vectors(&R, &C);
  DFPR_CUDA(cudaMemcpyAsync(snap.p, R, r_bytes, cudaMemcpyDeviceToDevice, s));
  DFPR_CUDA(cudaMemcpyAsync(snap.p + r_bytes, C, c_bytes, cudaMemcpyDeviceToDevice, s));
  const double d_before = g->d_before;
  const bool d_valid = g->d_before_valid;
  auto restore = [&]() {
    void *R2, *C2;
    vectors(&R2, &C2);
    DFPR_CUDA(cudaMemcpyAsync(R2, snap.p, r_bytes, cudaMemcpyDeviceToDevice, s));
    DFPR_CUDA(cudaMemcpyAsync(C2, snap.p + r_bytes, c_bytes, cudaMemcpyDeviceToDevice, s));
    g->pend.n_src = n_src;  // the pending arrays are left intact by an update
    g->pend.n_dst = n_dst;
    g->d_before = d_before;
    g->d_before_valid = d_valid;
  };
  cudaEvent_t e0, e1;
  DFPR_CUDA(cudaEventCreate(&e0));
  DFPR_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } guard{e0, e1};
  double best = INFINITY;
  int32_t bi = 0;
  for (int32_t i = 0; i < k; ++i) {
    if (i > 0) restore();
    dfpr_params q = plan_params(i);
    dfpr_stats st;
    DFPR_CUDA(cudaEventRecord(e0, s));
    const dfpr_status r = run_update(g, &q, &st, kRunDF);
    DFPR_CUDA(cudaEventRecord(e1, s));
    DFPR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    DFPR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double t = r == DFPR_OK ? (double)ms : INFINITY;
    if (trial_ms) trial_ms[i] = t;
    if (t < best) {
      best = t;
      bi = i;
    }
  }
  restore();
  *p = plan_params(bi);
  dfpr_stats st;
  const dfpr_status r = run_update(g, p, &st, kRunDF);
  if (stats) *stats = st;
  DFPR_CUDA(cudaStreamSynchronize(s));
  return r;
}

}  // namespace

dfpr_status dfpr_autotune(dfpr_graph* g, dfpr_params* p, int32_t n_candidates,
                          const int32_t* candidates, double* trial_ms, dfpr_stats* stats) {
  static const int32_t kDefaultPairs[8] = {2048, 2048, 4096, 8192, 8192, 8192, 16384, 16384};
  if (!g || !p || (candidates && n_candidates < 1)) {
    set_error("dfpr_autotune: need a graph, parameters and at least one candidate");
    return DFPR_EINVAL;
  }
  const int32_t* cand = candidates ? candidates : kDefaultPairs;
  const int32_t k = candidates ? n_candidates : 4;
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  DFPR_REQUIRE(p->mode != DFPR_MODE_JACOBI, DFPR_EINVAL,
               "dfpr_autotune: the split thresholds apply to the worklist and round schedules");
  std::vector<int32_t> plans((size_t)4 * k);
  for (int32_t i = 0; i < k; ++i) {
    plans[4 * i] = p->mode;
    plans[4 * i + 1] = p->grid_ctas;
    plans[4 * i + 2] = cand[2 * i];
    plans[4 * i + 3] = cand[2 * i + 1];
  }
  return autotune_plans(g, p, k, plans.data(), trial_ms, stats);
  API_END
}

dfpr_status dfpr_autotune_plans(dfpr_graph* g, dfpr_params* p, int32_t n_plans,
                                const int32_t* plans, int32_t* n_run, int32_t* plans_run,
                                double* trial_ms, dfpr_stats* stats) {
  if (n_run) *n_run = 0;
  if (!g || !p || (plans && n_plans < 1)) {
    set_error("dfpr_autotune_plans: need a graph, parameters and at least one plan");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  std::vector<int32_t> def;
  if (!plans) {
    // size classes (worklist grid: the graph's own rule, half of it, a full
    // wave of the occupancy limit),
    // degree classes (split thresholds), and the barrier-based schedule
    const int rule = default_worklist_grid(g, *p);
    dfpr_params q = *p;
    q.grid_ctas = 0;
    q.mode = DFPR_MODE_JACOBI;
    const int full = full_worklist_grid(g, *p);
    if (g->cfg.dead_end == DFPR_TELEPORT) {
      def = {DFPR_MODE_JACOBI, 0, 0, 0};
    } else {
      def = {DFPR_MODE_WORKLIST, rule, 0, 0,
             DFPR_MODE_WORKLIST, std::max(8, rule / 2), 0, 0,
             DFPR_MODE_WORKLIST, std::max(rule, full), 0, 0,
             DFPR_MODE_WORKLIST, rule, 2048, 2048,
             DFPR_MODE_WORKLIST, rule, 16384, 16384,
             DFPR_MODE_JACOBI, 0, 0, 0};
      // splits below the graph's minimum are left out, and so are repeats
      // (the rule's grid is a full wave on small devices)
      const long long min_split = std::max<long long>(256, (g->m + (1ll << 20) - 1) >> 20);
      std::vector<int32_t> keep;
      for (size_t i = 0; i < def.size(); i += 4) {
        if ((def[i + 2] != 0 && def[i + 2] < min_split) || (def[i + 3] != 0 && def[i + 3] < min_split))
          continue;
        bool seen = false;
        for (size_t j = 0; j < keep.size() && !seen; j += 4)
          seen = std::equal(keep.begin() + j, keep.begin() + j + 4, def.begin() + i);
        if (!seen) keep.insert(keep.end(), def.begin() + i, def.begin() + i + 4);
      }
      def.swap(keep);
    }
    plans = def.data();
    n_plans = (int32_t)(def.size() / 4);
  }
  if (n_run) *n_run = n_plans;
  if (plans_run) std::copy(plans, plans + 4 * n_plans, plans_run);
  return autotune_plans(g, p, n_plans, plans, trial_ms, stats);
  API_END
}

dfpr_status dfpr_nd_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  return run_update(g, p, stats, kRunND);
  API_END
}

dfpr_status dfpr_static_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats) {
  if (!g) {
    set_error("graph is NULL");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  return run_update(g, p, stats, kRunStatic);
  API_END
}

dfpr_status dfpr_residual(const dfpr_graph* gc, double alpha, double* linf, double* linf_rel) {
  if (!gc || !linf) {
    set_error("dfpr_residual: NULL argument");
    return DFPR_EINVAL;
  }
  if (!(alpha > 0.0 && alpha < 1.0)) {
    set_error("dfpr_residual: need 0 < alpha < 1");
    return DFPR_EINVAL;
  }
  dfpr_graph* g = const_cast<dfpr_graph*>(gc);
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  double a = 0.0, b = 0.0;
  residual(g, alpha, &a, &b);
  *linf = a;
  if (linf_rel) *linf_rel = b;
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_get_ranks(const dfpr_graph* gc, double* out, int on_device) {
  if (!gc || !out) {
    set_error("dfpr_get_ranks: NULL argument");
    return DFPR_EINVAL;
  }
  dfpr_graph* g = const_cast<dfpr_graph*>(gc);
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  const long long n = g->n;
  const int32_t* perm = g->relabeled ? g->perm.p : nullptr;
  if (g->cfg.precision == DFPR_FP64 && !perm) {
    DFPR_CUDA(cudaMemcpyAsync(out, g->R64.p, sizeof(double) * n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  } else {
    double* dst = out;
    bool stage = false;
    if (!on_device) {
      // page-locked host memory that the device can address is written by
      // the kernel itself; other host memory goes through a staging vector
      // kept with the graph
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
          attr.devicePointer) {
        dst = static_cast<double*>(attr.devicePointer);
      } else {
        cudaGetLastError();  // an unregistered pointer is not an error here
        if (g->rank_stage.count < (size_t)n) g->rank_stage.reset((size_t)n, s);
        dst = g->rank_stage.p;
        stage = true;
      }
    }
    if (g->cfg.precision == DFPR_FP64)
      k_ranks_out<double><<<blocks_for(n, kNT, sm_cap(16u)), kNT, 0, s>>>(g->R64.p, perm, dst, n);
    else
      k_ranks_out<float><<<blocks_for(n, kNT, sm_cap(16u)), kNT, 0, s>>>(g->R32.p, perm, dst, n);
    DFPR_LAUNCHED();
    if (stage)
      DFPR_CUDA(cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  }
  DFPR_CUDA(cudaStreamSynchronize(s));
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_set_ranks(dfpr_graph* g, const double* ranks, int on_device) {
  if (!g || !ranks) {
    set_error("dfpr_set_ranks: NULL argument");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  const long long n = g->n;
  const int32_t* perm = g->relabeled ? g->perm.p : nullptr;
  if (g->cfg.precision == DFPR_FP64 && !perm) {
    DFPR_CUDA(cudaMemcpyAsync(g->R64.p, ranks, sizeof(double) * n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {
    DevArray<double> tmp;
    const double* srcp = stage_in(g, tmp, ranks, n, on_device);
    if (g->cfg.precision == DFPR_FP64)
      k_ranks_in<double><<<blocks_for(n, kNT, sm_cap(16u)), kNT, 0, s>>>(srcp, perm, g->R64.p, n);
    else
      k_ranks_in<float><<<blocks_for(n, kNT, sm_cap(16u)), kNT, 0, s>>>(srcp, perm, g->R32.p, n);
    DFPR_LAUNCHED();
  }
  refresh_contributions(g);
  g->d_before_valid = false;  // new ranks: their dead-end mass is taken at the next batch
  DFPR_CUDA(cudaStreamSynchronize(s));
  return DFPR_OK;
  API_END
}

static dfpr_status export_dir(const dfpr_graph* gc, bool csr, int64_t* offsets, int32_t* idx,
                              int on_device) {
  if (!gc || !offsets || !idx) {
    set_error("dfpr_get_csr/csc: NULL argument");
    return DFPR_EINVAL;
  }
  dfpr_graph* g = const_cast<dfpr_graph*>(gc);
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  DevArray<long long> toff;
  DevArray<int32_t> tidx;
  long long* doff = (long long*)offsets;
  int32_t* didx = idx;
  if (!on_device) {
    toff.reset((size_t)g->n + 1, s);
    tidx.reset((size_t)g->m + 1, s);
    doff = toff.p;
    didx = tidx.p;
  }
  graph_export(g, csr ? g->out : g->in, doff, didx);
  if (!on_device) {
    DFPR_CUDA(cudaMemcpyAsync(offsets, doff, sizeof(long long) * (g->n + 1), cudaMemcpyDeviceToHost, s));
    DFPR_CUDA(cudaMemcpyAsync(idx, didx, sizeof(int32_t) * g->m, cudaMemcpyDeviceToHost, s));
  }
  DFPR_CUDA(cudaStreamSynchronize(s));
  return DFPR_OK;
  API_END
}

dfpr_status dfpr_get_csr(const dfpr_graph* g, int64_t* offsets, int32_t* idx, int on_device) {
  return export_dir(g, true, offsets, idx, on_device);
}

dfpr_status dfpr_get_csc(const dfpr_graph* g, int64_t* offsets, int32_t* idx, int on_device) {
  return export_dir(g, false, offsets, idx, on_device);
}

dfpr_status dfpr_initial_affected(dfpr_graph* g, uint8_t* affected, int on_device, int64_t* count) {
  if (count) *count = 0;
  if (!g || !affected) {
    set_error("dfpr_initial_affected: NULL argument");
    return DFPR_EINVAL;
  }
  API_BEGIN
  BusyGuard bg(g);
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  DevArray<uint8_t> tmp;
  uint8_t* dst = affected;
  if (!on_device) {
    tmp.reset((size_t)g->n, s);
    dst = tmp.p;
  }
  long long c = 0;
  initial_affected(g, dst, &c);
  if (!on_device)
    DFPR_CUDA(cudaMemcpyAsync(affected, dst, (size_t)g->n, cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaStreamSynchronize(s));
  if (count) *count = c;
  return DFPR_OK;
  API_END
}

}  // extern "C"
