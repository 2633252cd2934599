// Serving runtime: a thread that keeps a graph (set) resident and serves
// update requests in cycles; each cycle applies every admitted request's batch
// and updates all affected graphs with one persistent launch (see dfpr.h).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "df.cuh"
#include "graph.cuh"

namespace dfpr {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int32_t part = 0;
  std::vector<int32_t> ds, dd, is, id_;
  double submit_ms = 0, admit_ms = 0, done_ms = 0;
  int64_t cycle = -1;
  int32_t cycle_requests = 0;
  dfpr_status status = DFPR_OK;
  bool done = false;
  int64_t edges() const { return (int64_t)ds.size() + (int64_t)is.size(); }
};

// Device bytes a cycle needs per batch edge: batch keys and their sort buffer,
// flags and positions, real-change lists in both orders, row-merge plans.
constexpr double kBytesPerBatchEdge = 160.0;

}  // namespace
}  // namespace dfpr

struct dfpr_server {
  dfpr_graph* g = nullptr;
  dfpr_params p;
  int32_t max_slots = 64;
  double mem_fraction = 0.5;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<dfpr::Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<dfpr::Request>> requests;
  int64_t next_id = 1;
  int64_t cycles = 0;
  bool in_cycle = false;
  bool stop = false;
  std::thread th;
  dfpr::DevArray<int32_t> dev_batch;  // the cycle's batch arrays on the device
  std::vector<int32_t> host_batch;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace dfpr {
namespace {

// Applies one layer of requests (at most one per graph) as one batch.
void apply_layer(dfpr_server* s, const std::vector<std::shared_ptr<Request>>& layer) {
  dfpr_graph* g = s->g;
  int64_t nd = 0, ni = 0;
  for (auto& r : layer) {
    nd += (int64_t)r->ds.size();
    ni += (int64_t)r->is.size();
  }
  if (nd + ni == 0) return;
  // host staging: del_src | del_dst | ins_src | ins_dst in global ids
  s->host_batch.resize((size_t)(2 * (nd + ni)));
  int32_t* ds = s->host_batch.data();
  int32_t* dd = ds + nd;
  int32_t* is = dd + nd;
  int32_t* id = is + ni;
  int64_t od = 0, oi = 0;
  for (auto& r : layer) {
    const int32_t base = g->nparts > 1 ? g->part_off_host[r->part] : 0;
    for (size_t k = 0; k < r->ds.size(); ++k) {
      ds[od + k] = r->ds[k] + base;
      dd[od + k] = r->dd[k] + base;
    }
    for (size_t k = 0; k < r->is.size(); ++k) {
      is[oi + k] = r->is[k] + base;
      id[oi + k] = r->id_[k] + base;
    }
    od += (int64_t)r->ds.size();
    oi += (int64_t)r->is.size();
  }
  s->dev_batch.ensure((size_t)(2 * (nd + ni)), g->stream);
  DFPR_CUDA(cudaMemcpyAsync(s->dev_batch.p, ds, sizeof(int32_t) * 2 * (nd + ni),
                            cudaMemcpyHostToDevice, g->stream));
  const int32_t* d = s->dev_batch.p;
  long long applied[2] = {0, 0};
  graph_apply(g, d, d + nd, nd, d + 2 * nd, d + 2 * nd + ni, ni, applied);
}

void serve(dfpr_server* s) {
  cudaSetDevice(s->g->device);
  while (true) {
    std::vector<std::shared_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->queue.empty()) break;  // stop requested and nothing left
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
      }
      const double budget = s->mem_fraction * (double)free_b;
      double need = 0;
      while (!s->queue.empty() && (int32_t)admitted.size() < s->max_slots) {
        auto& r = s->queue.front();
        const double b = kBytesPerBatchEdge * (double)r->edges();
        if (!admitted.empty() && need + b > budget) break;  // memory admission
        need += b;
        admitted.push_back(r);
        s->queue.pop_front();
      }
      s->in_cycle = true;
    }
    const double t_admit = s->now_ms();
    dfpr_status st = DFPR_OK;
    try {
      // layers: the k-th request of each graph goes to layer k, so requests
      // for one graph apply in arrival order
      std::unordered_map<int32_t, int> seen;
      std::vector<std::vector<std::shared_ptr<Request>>> layers;
      for (auto& r : admitted) {
        const int k = seen[r->part]++;
        if ((int)layers.size() <= k) layers.resize(k + 1);
        layers[k].push_back(r);
      }
      for (auto& layer : layers) apply_layer(s, layer);
      dfpr_stats stats;
      st = run_update(s->g, &s->p, &stats, kRunDF);
    } catch (const Fail& f) {
      st = f.st;
    } catch (...) {
      st = DFPR_ECUDA;
    }
    const double t_done = s->now_ms();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& r : admitted) {
        r->admit_ms = t_admit;
        r->done_ms = t_done;
        r->status = st;
        r->cycle = s->cycles;
        r->cycle_requests = (int32_t)admitted.size();
        r->done = true;
      }
      ++s->cycles;
      s->in_cycle = false;
    }
    s->cv_done.notify_all();
  }
}

bool ids_ok(const int32_t* a, int64_t n, int32_t lim) {
  for (int64_t i = 0; i < n; ++i)
    if (a[i] < 0 || a[i] >= lim) return false;
  return true;
}

}  // namespace
}  // namespace dfpr

using namespace dfpr;

extern "C" {

dfpr_status dfpr_server_create(dfpr_graph* g, const dfpr_params* p, int32_t max_slots,
                               double mem_fraction, dfpr_server** out) {
  if (out) *out = nullptr;
  if (!g || !out || max_slots < 1 || !(mem_fraction > 0.0 && mem_fraction <= 1.0)) {
    set_error("dfpr_server_create: need a graph, max_slots >= 1 and 0 < mem_fraction <= 1");
    return DFPR_EINVAL;
  }
  int z = 0;
  if (!g->busy.compare_exchange_strong(z, 1)) {
    set_error("dfpr_server_create: another call on this graph is in progress");
    return DFPR_EBUSY;
  }
  dfpr_server* s = nullptr;
  try {
    s = new dfpr_server();
  } catch (...) {
    g->busy.store(0);
    set_error("host allocation failed");
    return DFPR_ENOMEM;
  }
  s->g = g;
  if (p) s->p = *p;
  else dfpr_default_params(&s->p);
  s->max_slots = max_slots;
  s->mem_fraction = mem_fraction;
  s->t0 = Clock::now();
  try {
    s->th = std::thread(serve, s);
  } catch (...) {
    g->busy.store(0);
    delete s;
    set_error("dfpr_server_create: could not start the server thread");
    return DFPR_ENOMEM;
  }
  *out = s;
  return DFPR_OK;
}

dfpr_status dfpr_server_submit(dfpr_server* s, int32_t part, int64_t n_del, const int32_t* del_src,
                               const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                               const int32_t* ins_dst, int64_t* request_id) {
  if (request_id) *request_id = 0;
  if (!s || part < 0 || part >= s->g->nparts || n_del < 0 || n_ins < 0 ||
      (n_del > 0 && (!del_src || !del_dst)) || (n_ins > 0 && (!ins_src || !ins_dst))) {
    set_error("dfpr_server_submit: invalid arguments");
    return DFPR_EINVAL;
  }
  const int32_t lim = s->g->nparts > 1
                          ? s->g->part_off_host[part + 1] - s->g->part_off_host[part]
                          : s->g->n;
  if (!ids_ok(del_src, n_del, lim) || !ids_ok(del_dst, n_del, lim) || !ids_ok(ins_src, n_ins, lim) ||
      !ids_ok(ins_dst, n_ins, lim)) {
    set_error("dfpr_server_submit: a vertex id is outside its graph");
    return DFPR_EINVAL;
  }
  std::shared_ptr<Request> r;
  try {
    r = std::make_shared<Request>();
    r->part = part;
    r->ds.assign(del_src, del_src + n_del);
    r->dd.assign(del_dst, del_dst + n_del);
    r->is.assign(ins_src, ins_src + n_ins);
    r->id_.assign(ins_dst, ins_dst + n_ins);
  } catch (...) {
    set_error("host allocation failed");
    return DFPR_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("dfpr_server_submit: the server is stopping");
      return DFPR_EBUSY;
    }
    r->id = s->next_id++;
    r->submit_ms = s->now_ms();
    s->requests[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  if (request_id) *request_id = r->id;
  return DFPR_OK;
}

dfpr_status dfpr_server_wait(dfpr_server* s, int64_t request_id, dfpr_request_info* info) {
  if (!s) {
    set_error("dfpr_server_wait: server is NULL");
    return DFPR_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) {
    set_error("dfpr_server_wait: unknown request id");
    return DFPR_EINVAL;
  }
  std::shared_ptr<Request> r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  if (info) {
    info->status = r->status;
    info->cycle_requests = r->cycle_requests;
    info->cycle = r->cycle;
    info->submit_ms = r->submit_ms;
    info->admit_ms = r->admit_ms;
    info->done_ms = r->done_ms;
  }
  s->requests.erase(request_id);
  return DFPR_OK;
}

dfpr_status dfpr_server_drain(dfpr_server* s) {
  if (!s) {
    set_error("dfpr_server_drain: server is NULL");
    return DFPR_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->queue.empty() && !s->in_cycle; });
  return DFPR_OK;
}

dfpr_status dfpr_server_destroy(dfpr_server* s) {
  if (!s) return DFPR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  dfpr_graph* g = s->g;
  {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    s->dev_batch.release();
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete s;
  g->busy.store(0);
  return DFPR_OK;
}

}  // extern "C"
