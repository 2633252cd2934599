// Internal definitions shared by the translation units of libdfpr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/dfpr.h"

namespace dfpr {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

void set_error(const std::string& msg);
const char* get_error();

struct Fail {
  dfpr_status st;
};

#define DFPR_CUDA(call)                                                          \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::dfpr::set_error(std::string(#call) + ": " + cudaGetErrorString(e_) +     \
                        " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
      throw ::dfpr::Fail{DFPR_ECUDA};                                            \
    }                                                                            \
  } while (0)

#define DFPR_REQUIRE(cond, code, msg)   \
  do {                                  \
    if (!(cond)) {                      \
      ::dfpr::set_error(msg);           \
      throw ::dfpr::Fail{code};         \
    }                                   \
  } while (0)

// Kernel launches issued by the library (a process-wide counter).
extern std::atomic<long long> g_launches;

// Launch-error check after a kernel launch; also counts the launch.
#define DFPR_LAUNCHED()                                   \
  do {                                                    \
    ::dfpr::g_launches.fetch_add(1, std::memory_order_relaxed); \
    DFPR_CUDA(cudaGetLastError());                        \
  } while (0)

// ---------------------------------------------------------------------------
// Device memory (through the installable allocator)
// ---------------------------------------------------------------------------

// The free routine that matches an allocation (captured when it was made).
struct FreeRec {
  dfpr_free_fn fn;
  void* ctx;
};
void* dev_alloc(size_t bytes, cudaStream_t s, FreeRec* rec);  // throws Fail{ENOMEM}
void dev_free(void* p, size_t bytes, cudaStream_t s, const FreeRec& rec);

template <class T>
struct DevArray {
  T* p = nullptr;
  size_t count = 0;
  cudaStream_t s = nullptr;
  FreeRec rec{nullptr, nullptr};
  void reset(size_t n, cudaStream_t st) {
    release();
    s = st;
    if (n) p = (T*)dev_alloc(n * sizeof(T), st, &rec);
    count = n;
  }
  // Grows to at least n elements (contents are not preserved).
  void ensure(size_t n, cudaStream_t st) {
    if (n > count) reset(n + n / 4 + 64, st);
  }
  void release() {
    if (p) dev_free(p, count * sizeof(T), s, rec);
    p = nullptr;
    count = 0;
  }
  DevArray() = default;
  DevArray(const DevArray&) = delete;
  DevArray& operator=(const DevArray&) = delete;
  ~DevArray() { release(); }
};

// Scratch arena: numbered buffers that grow on demand (contents are not
// preserved across growth). Slot numbers are assigned in graph.cu / df.cu /
// primitives.cuh so that nested users never share a slot.
struct Scratch {
  DevArray<unsigned char> buf[40];
  template <class T>
  T* get(int slot, size_t n, cudaStream_t s) {
    buf[slot].ensure(n * sizeof(T) + 16, s);
    return (T*)buf[slot].p;
  }
};

// ---------------------------------------------------------------------------
// Graph layout
// ---------------------------------------------------------------------------

// Per-vertex record of one worklist call (built at its start, ranks copied
// back at its end): the rank, the rank at the last expansion, the in-row as
// offset << 25 | degree, the out-degree and a flag word (bit 0: recomputed in
// this call). 32 bytes, one sector, so a recomputation reads its vertex's
// state in one random access.
struct __align__(32) VRec {
  unsigned long long a;   // FP64: rank bits; FP32: rank bits | x bits << 32
  unsigned long long b;   // FP64: x bits;    FP32: out-degree | flags << 32
  unsigned long long in;  // in-row offset << 25 | in-degree
  unsigned long long c;   // FP64: out-degree | flags << 32; FP32: unused
};

// One row of CSR or CSC: edges[off .. off + deg) hold the row, sorted; the
// slot reserves cap >= deg entries so that batches update it in place.
struct __align__(16) RowDesc {
  long long off;
  int deg;
  int cap;
};

struct Rows {
  DevArray<RowDesc> rows;          // n
  DevArray<int32_t> edges;         // ecap
  long long ecap = 0;              // capacity of edges
  DevArray<unsigned long long> tail;  // 1: next free position of the spare area
};

// A counter alone on its own 256-byte line: the queue counters are hit by
// every warp, and counters sharing a line would serialise at one L2 slice.
struct __align__(256) HotU64 {
  unsigned long long v;
  unsigned long long pad_[31];
};
struct __align__(256) HotI64 {
  long long v;
  long long pad_[31];
};

// Device control block of one rank iteration (all counters 64-bit).
struct DfCtl {
  HotU64 head;        // queue positions claimed by consumers
  HotU64 tail;        // queue positions claimed by producers
  HotI64 avail;       // pushed but not yet claimed
  HotI64 pending;     // queued + running vertices + open marking items
  HotU64 mark_next;   // next marking item to claim
  HotU64 processed;   // recomputations (work cap)
  HotI64 len;         // affected-list length (round / jacobi)
  HotI64 nc;          // vertices flagged not converged (round)
  HotU64 thead;       // token ring (chunks of heavy gathers and of marking): consumers
  HotU64 ttail;       //   producers
  HotI64 tavail;      //   published, not yet claimed
  HotI64 open_tokens; // round: gather tokens published and not yet summed
  HotU64 fhead;       // free ring of heavy-gather job slots: consumers
  HotU64 ftail;       //   producers
  HotI64 favail;      //   free slots
  unsigned long long n_src_items;  // marking items over out-rows of sources
  unsigned long long n_items;      // all marking items
  long long n_mark_dst;            // deletion targets to mark
  unsigned int status;             // 0, or the dfpr_status that stopped the workers
  unsigned int abort;              // 1: workers stop
  unsigned long long edges, expansions, edges_marked, pushes, affected;
  unsigned long long max_change_bits;  // max |change| of a recomputation (bits of a double)
  long long nheavy;                // jacobi: long in-rows registered this iteration
  long long heavy_chunks;          // jacobi: their gather_split-edge chunks
  long long work_cap;              // cap on recomputations (worklist)
  unsigned long long t_start;      // globaltimer at launch
  double dsum;                     // rank held by dead ends (teleport)
  unsigned long long passes;       // round: passes reached
  unsigned long long batches;      // worklist: batches taken from the queue
  unsigned long long tokens;       // worklist: chunk tokens processed
  unsigned long long jobs;         // worklist: heavy gathers split into chunk tokens
  unsigned long long phase[5];     // worklist: cycles idle, claim, gather, expand, finish
};

struct Pending {
  DevArray<int32_t> src;   // sources of real changes (marking: out-rows)
  DevArray<int32_t> dst;   // targets of real deletions
  long long n_src = 0, n_dst = 0;
};

// Contribution C[u] = R[u] / |out(u)| of a vertex, as stored for gathers.
// FP64 graphs keep it as a 64-bit fixed-point number with scale 2^60, so a
// gather sums exactly with integer adds (GB300's FP64 rate is a small
// fraction of its integer and FP32 rates): each term is rounded once, to
// 2^-61 absolute, and a sum stays below 8. Ranks never exceed 1 (the worklist
// epilogue clamps transients there), so every term is at most 1 and a
// vertex's in-sum reaches 8 only with more than 8 in-neighbours at rank 1,
// i.e. a rank mass eight times the graph's total of 1.
// FP32 graphs keep the float quotient.
constexpr double kFix = 1152921504606846976.0;          // 2^60
constexpr double kInvFix = 1.0 / 1152921504606846976.0;  // 2^-60
__device__ __forceinline__ long long contrib_of(double r, int d) {
  return d > 0 ? __double2ll_rn((r / (double)d) * kFix) : 0ll;
}
__device__ __forceinline__ float contrib_of(float r, int d) {
  return d > 0 ? __fdiv_rn(r, (float)d) : 0.f;
}

// Graph of vertex v in a set of k graphs with vertex offsets off[0..k]
// (binary search; off[0] = 0 <= v < off[k]).
__device__ __forceinline__ int part_of(const int32_t* __restrict__ off, int k, int v) {
  int lo = 0, hi = k;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= v) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace dfpr

struct dfpr_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int32_t n = 0;
  int bits = 1;             // ids fit in `bits` bits
  long long m = 0;          // live edges (both directions hold m)
  long long last_real_del = 0;  // real deletions of the batch being applied
  // teleport graphs: dead-end mass of the ranks before the first batch applied
  // since the ranks were last computed or set (the D those ranks were
  // computed with); d_before_valid is false when no batch is pending
  double d_before = 0.0;
  bool d_before_valid = false;
  dfpr_graph_config cfg;
  dfpr::Rows out, in;
  // ranks: FP64 or FP32 arrays (one of each pair is used)
  dfpr::DevArray<double> R64;              // rank
  dfpr::DevArray<long long> C64;           // contribution R/outdeg, fixed point 2^-60
  dfpr::DevArray<float> R32, C32;
  dfpr::DevArray<dfpr::VRec> vrec;        // worklist: per-vertex records of the running call
  dfpr::DevArray<unsigned long long> hold;  // worklist: per-warp hold records (helping)
  dfpr::DevArray<double> rank_stage;         // get_ranks into pageable host memory
  dfpr::DevArray<int32_t> jh_v;             // jacobi: long in-rows of an iteration (vertex,
  dfpr::DevArray<int32_t> jh_rem;           //   chunks not yet summed,
  dfpr::DevArray<unsigned long long> jh_sum;  //   partial sums,
  dfpr::DevArray<long long> jh_off;         //   chunk offsets)
  dfpr::DevArray<double> R64b;             // second vectors of the Jacobi schedule
  dfpr::DevArray<long long> C64b;
  dfpr::DevArray<float> R32b, C32b;
  dfpr::DevArray<uint32_t> state;         // 2 bits per vertex: bit0 queued, bit1 running
  dfpr::DevArray<int32_t> queue;          // qcap slots, -1 when empty
  unsigned long long qcap = 0;
  dfpr::DevArray<unsigned long long> tokens;  // token ring, all ones when empty
  unsigned long long tcap = 0;
  dfpr::DevArray<int32_t> job_ring;       // free job slots, -1 when empty
  dfpr::DevArray<int32_t> job_v;          // vertex of a job slot
  dfpr::DevArray<int32_t> job_rem;        // chunks of the job not yet summed
  dfpr::DevArray<unsigned long long> job_sum;  // partial sums (fixed point, or FP64 bits)
  int jcap = 0;
  dfpr::DevArray<dfpr::DfCtl> ctl;
  dfpr::DevArray<int32_t> affected_list;  // round mode: affected vertices in marking order
  dfpr::DevArray<uint32_t> va_bits;       // round mode: affected bitmap
  dfpr::DevArray<uint32_t> rc_bits;       // round mode: not-converged bitmap
  dfpr::DevArray<unsigned long long> pass_ctr;  // round mode: per-pass claim counters
  dfpr::DevArray<uint32_t> item_done;     // round mode: marking items completed (helping)
  int nparts = 1;                         // graphs in the set (disjoint union)
  dfpr::DevArray<int32_t> part_off;       // nparts + 1 vertex offsets (when nparts > 1)
  dfpr::DevArray<unsigned long long> part_done;  // per graph: last recomputation end (globaltimer)
  std::vector<int32_t> part_off_host;
  std::vector<double> part_ms;            // completion times of the last worklist update
  dfpr::DevArray<int32_t> perm;           // caller id -> internal id (when reordered)
  dfpr::DevArray<int32_t> iperm;          // internal id -> caller id
  bool relabeled = false;
  long long max_degree = -1;              // largest in- or out-degree, when tracked
  dfpr::Pending pend;
  dfpr::Scratch scratch;
  dfpr::DevArray<unsigned long long> host_sync;  // small device words read back
  unsigned long long* pinned = nullptr;   // pinned host words for read-back
  std::atomic<int> busy{0};
  std::vector<cudaStream_t> retired_streams;  // owned streams replaced by set_stream,
                                              // destroyed with the graph
  int sm_count = 0;
  int max_ctas = 0;
  // CUDA-graph replay of the DF update's device work (dfpr_graph_set_capture)
  bool capture = false;
  cudaGraphExec_t cap_exec = nullptr;
  std::vector<unsigned char> cap_key;       // what the captured launches depend on
  cudaEvent_t cap_ev[2] = {nullptr, nullptr};
  unsigned long long* cap_host = nullptr;   // pinned: pending counts read at replay
  dfpr::DevArray<long long> cap_dev;        // 2: the same counts on the device
  dfpr::Scratch cap_scratch;                // marking items and their scan, capture only
  long long cap_launches = 0;               // kernels in the captured graph
  long long cap_captures = 0, cap_replays = 0;
};
