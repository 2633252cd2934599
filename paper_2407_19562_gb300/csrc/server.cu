// Serving runtime with continuous batching. A server owns one or more
// resident units (a graph, or a set of graphs from dfpr_graph_load_parts),
// each with its own stream and one worker thread. A unit's worker admits the
// unit's queued requests whenever the unit is idle and the server has free
// slots and memory, applies them, and runs one update over the unit (one
// persistent launch for every admitted request of that unit). Units update
// independently, so a request for an idle unit is admitted at once even while
// other units' updates are on the GPU, and their launches overlap on the
// device. A unit never changes while its own update reads it (read-only
// snapshot, Sec. 3.4): requests that arrive for a busy unit join its next
// update.
#include <cuda_runtime.h>

#include <algorithm>
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
  int32_t unit = 0;  // the unit that holds the graph
  int32_t part = 0;  // the graph's index within its unit
  std::vector<int32_t> ds, dd, is, id_;
  double submit_ms = 0, admit_ms = 0, done_ms = 0;
  int64_t cycle = -1;
  int32_t cycle_requests = 0;
  dfpr_status status = DFPR_OK;
  bool done = false;
  int64_t edges() const { return (int64_t)ds.size() + (int64_t)is.size(); }
};

// Device bytes an update needs per batch edge: batch keys and their sort
// buffer, flags and positions, real-change lists in both orders, row-merge plans.
constexpr double kBytesPerBatchEdge = 160.0;

struct Unit {
  dfpr_graph* g = nullptr;
  std::deque<std::shared_ptr<Request>> queue;
  bool running = false;
  std::thread th;
  DevArray<int32_t> dev_batch;  // the update's batch arrays on the device
  std::vector<int32_t> host_batch;
};

}  // namespace
}  // namespace dfpr

struct dfpr_server {
  std::vector<std::unique_ptr<dfpr::Unit>> units;
  std::vector<int32_t> part_unit, part_local;  // global part -> (unit, part within it)
  dfpr_params p;
  int32_t max_slots = 64;
  double mem_fraction = 0.5;
  int grid_share = 0;  // CTAs per launch when units update concurrently (0: full grid)
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<int64_t, std::shared_ptr<dfpr::Request>> requests;
  int64_t next_id = 1;
  int64_t cycles = 0;
  int32_t in_flight = 0;    // admitted requests not yet done
  int32_t queued = 0;       // requests waiting in unit queues
  double reserved = 0.0;    // batch bytes of admitted requests
  bool stop = false;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace dfpr {
namespace {

// Applies one layer of requests (at most one per graph of the unit) as one batch.
void apply_layer(Unit* u, const std::vector<std::shared_ptr<Request>>& layer) {
  dfpr_graph* g = u->g;
  int64_t nd = 0, ni = 0;
  for (auto& r : layer) {
    nd += (int64_t)r->ds.size();
    ni += (int64_t)r->is.size();
  }
  if (nd + ni == 0) return;
  // host staging: del_src | del_dst | ins_src | ins_dst in the unit's global ids
  u->host_batch.resize((size_t)(2 * (nd + ni)));
  int32_t* ds = u->host_batch.data();
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
  u->dev_batch.ensure((size_t)(2 * (nd + ni)), g->stream);
  DFPR_CUDA(cudaMemcpyAsync(u->dev_batch.p, ds, sizeof(int32_t) * 2 * (nd + ni),
                            cudaMemcpyHostToDevice, g->stream));
  const int32_t* d = u->dev_batch.p;
  long long applied[2] = {0, 0};
  graph_apply(g, d, d + nd, nd, d + 2 * nd, d + 2 * nd + ni, ni, applied);
}

// Worker of one unit: admission, update, completion, until the server stops
// and the unit's queue is empty.
void serve_unit(dfpr_server* s, Unit* u) {
  cudaSetDevice(u->g->device);
  while (true) {
    std::vector<std::shared_ptr<Request>> admitted;
    double need = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return (s->stop && u->queue.empty()) ||
               (!u->queue.empty() && s->in_flight < s->max_slots);
      });
      if (u->queue.empty()) break;  // stop requested and nothing left
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
      }
      const double budget = s->mem_fraction * (double)free_b - s->reserved;
      while (!u->queue.empty() && s->in_flight + (int32_t)admitted.size() < s->max_slots) {
        auto& r = u->queue.front();
        const double b = kBytesPerBatchEdge * (double)r->edges();
        // memory admission; with nothing else in flight one request always goes
        if ((!admitted.empty() || s->in_flight > 0) && need + b > budget) break;
        need += b;
        admitted.push_back(r);
        u->queue.pop_front();
      }
      if (admitted.empty()) {  // no memory now (so another update is in flight): wait for it
        s->cv_work.wait(lk);
        continue;
      }
      s->in_flight += (int32_t)admitted.size();
      s->queued -= (int32_t)admitted.size();
      s->reserved += need;
      u->running = true;
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
      for (auto& layer : layers) apply_layer(u, layer);
      dfpr_params p = s->p;
      if (p.grid_ctas == 0 && s->grid_share > 0)
        p.grid_ctas = std::min(default_worklist_grid(u->g, p), s->grid_share);
      dfpr_stats stats;
      st = run_update(u->g, &p, &stats, kRunDF);
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
      s->in_flight -= (int32_t)admitted.size();
      s->reserved -= need;
      if (s->in_flight == 0) s->reserved = 0.0;  // no drift from rounding
      u->running = false;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // slots and memory are free again
  }
}

bool ids_ok(const int32_t* a, int64_t n, int32_t lim) {
  for (int64_t i = 0; i < n; ++i)
    if (a[i] < 0 || a[i] >= lim) return false;
  return true;
}

void release_units(dfpr_server* s) {
  for (auto& u : s->units) {
    if (!u->g) continue;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(u->g->device);
    u->dev_batch.release();
    if (prev >= 0) cudaSetDevice(prev);
    u->g->busy.store(0);
  }
}

}  // namespace
}  // namespace dfpr

using namespace dfpr;

extern "C" {

dfpr_status dfpr_server_create_units(int32_t k, dfpr_graph* const* units, const dfpr_params* p,
                                     int32_t max_slots, double mem_fraction, int32_t grid_share,
                                     dfpr_server** out) {
  if (out) *out = nullptr;
  if (k < 1 || !units || !out || max_slots < 1 || !(mem_fraction > 0.0 && mem_fraction <= 1.0) ||
      grid_share < 0) {
    set_error("dfpr_server_create: need k >= 1 units, max_slots >= 1, 0 < mem_fraction <= 1 "
              "and grid_share >= 0");
    return DFPR_EINVAL;
  }
  for (int32_t i = 0; i < k; ++i) {
    if (!units[i]) {
      set_error("dfpr_server_create: a unit is NULL");
      return DFPR_EINVAL;
    }
    for (int32_t j = 0; j < i; ++j)
      if (units[j] == units[i]) {
        set_error("dfpr_server_create: a unit is given twice");
        return DFPR_EINVAL;
      }
  }
  // take every unit, or none
  int32_t taken = 0;
  for (; taken < k; ++taken) {
    int z = 0;
    if (!units[taken]->busy.compare_exchange_strong(z, 1)) break;
  }
  if (taken < k) {
    for (int32_t j = 0; j < taken; ++j) units[j]->busy.store(0);
    set_error("dfpr_server_create: another call on a unit is in progress");
    return DFPR_EBUSY;
  }
  dfpr_server* s = nullptr;
  try {
    s = new dfpr_server();
    for (int32_t i = 0; i < k; ++i) {
      s->units.emplace_back(new Unit());
      s->units.back()->g = units[i];
      for (int32_t j = 0; j < units[i]->nparts; ++j) {
        s->part_unit.push_back(i);
        s->part_local.push_back(j);
      }
    }
  } catch (...) {
    for (int32_t j = 0; j < k; ++j) units[j]->busy.store(0);
    delete s;
    set_error("host allocation failed");
    return DFPR_ENOMEM;
  }
  if (p) s->p = *p;
  else dfpr_default_params(&s->p);
  s->max_slots = max_slots;
  s->mem_fraction = mem_fraction;
  s->grid_share = grid_share;
  s->t0 = Clock::now();
  size_t started = 0;
  try {
    for (; started < s->units.size(); ++started) {
      Unit* u = s->units[started].get();
      u->th = std::thread(serve_unit, s, u);
    }
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (size_t i = 0; i < started; ++i) s->units[i]->th.join();
    release_units(s);
    delete s;
    set_error("dfpr_server_create: could not start the worker threads");
    return DFPR_ENOMEM;
  }
  *out = s;
  return DFPR_OK;
}

dfpr_status dfpr_server_create(dfpr_graph* g, const dfpr_params* p, int32_t max_slots,
                               double mem_fraction, dfpr_server** out) {
  if (out) *out = nullptr;
  if (!g) {
    set_error("dfpr_server_create: need a graph");
    return DFPR_EINVAL;
  }
  return dfpr_server_create_units(1, &g, p, max_slots, mem_fraction, 0, out);
}

dfpr_status dfpr_server_submit(dfpr_server* s, int32_t part, int64_t n_del, const int32_t* del_src,
                               const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                               const int32_t* ins_dst, int64_t* request_id) {
  if (request_id) *request_id = 0;
  if (!s || part < 0 || part >= (int32_t)s->part_unit.size() || n_del < 0 || n_ins < 0 ||
      (n_del > 0 && (!del_src || !del_dst)) || (n_ins > 0 && (!ins_src || !ins_dst))) {
    set_error("dfpr_server_submit: invalid arguments");
    return DFPR_EINVAL;
  }
  const int32_t ui = s->part_unit[part], lp = s->part_local[part];
  const dfpr_graph* g = s->units[ui]->g;
  const int32_t lim = g->nparts > 1 ? g->part_off_host[lp + 1] - g->part_off_host[lp] : g->n;
  if (!ids_ok(del_src, n_del, lim) || !ids_ok(del_dst, n_del, lim) || !ids_ok(ins_src, n_ins, lim) ||
      !ids_ok(ins_dst, n_ins, lim)) {
    set_error("dfpr_server_submit: a vertex id is outside its graph");
    return DFPR_EINVAL;
  }
  std::shared_ptr<Request> r;
  try {
    r = std::make_shared<Request>();
    r->unit = ui;
    r->part = lp;
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
    s->units[ui]->queue.push_back(r);
    ++s->queued;
  }
  s->cv_work.notify_all();
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
  s->cv_done.wait(lk, [&] { return s->queued == 0 && s->in_flight == 0; });
  return DFPR_OK;
}

dfpr_status dfpr_server_destroy(dfpr_server* s) {
  if (!s) return DFPR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& u : s->units)
    if (u->th.joinable()) u->th.join();
  release_units(s);
  delete s;
  return DFPR_OK;
}

}  // extern "C"
