// Rank iterations of the Dynamic Frontier approach (arXiv 2407.19562, Sec. 4)
// and of the static / naive-dynamic baselines (Sec. 3.3, 3.5.1), on one GPU.
//
// Every schedule recomputes a vertex v with Eq. 1 as
//     r = (1 - alpha) / n + alpha * sum_{u in in(v)} C[u],   C[u] = R[u] / |out(u)|
// where C is kept next to R and refreshed whenever R[u] or |out(u)| changes,
// so a gather reads one id and one value per in-edge.
//
// Schedules:
//  * worklist (persistent kernel, no grid-wide barrier): vertices flagged
//    not-converged sit in a device queue; a warp pops up to 32, recomputes
//    them in place, marks out-neighbours when the rank moved by more than the
//    frontier tolerance in this recomputation (or has drifted by more than
//    ten times that since the vertex last marked them; FP32 mode uses the
//    drift rule alone), and re-queues itself while its change exceeds the
//    iteration tolerance. Each vertex has a 2-bit state (queued, running) so
//    that no vertex is recomputed by two warps at once and no update is lost.
//    In-rows and out-rows longer than a few thousand edges are cut into
//    tokens that any warp takes. The iteration ends when the count of queued
//    + running vertices + open marking items and tokens reaches zero.
//  * round (Alg. 2): every affected vertex is recomputed in every pass; warps
//    claim chunks of a pass from a per-pass counter and move to the next pass
//    without waiting; a per-vertex not-converged flag R_C and its count end
//    the iteration; marking uses the helping rule (unfinished marking items
//    are redone by idle warps); heavy in-rows are cut into gather tokens as
//    in the worklist.
//  * jacobi (Alg. 1 / Alg. 3 / Alg. 5): two vectors, one kernel per iteration,
//    L-inf reduction, swap; marks take effect from the next iteration.
//
// Every wait is bounded by the call's time budget (%globaltimer); on expiry
// the kernel records DFPR_ETIMEOUT and returns.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "df.cuh"
#include "graph.cuh"
#include "primitives.cuh"

namespace dfpr {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNT = 256;
constexpr int kWPB = kNT / 32;
constexpr int kMarkChunk = 1024;  // out-edges per marking item

// Scratch slots (see common.cuh; graph.cu uses 0..28).
enum { kSMarkCnt = 30, kSMarkOff = 31, kSListKeys = 32, kSListTmp = 33 };
constexpr int kJacobiChunk = 2048;  // in-edges per chunk of a long in-row (jacobi schedule)

#define GRID_STRIDE(i, n)                                                             \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
       i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ long long ld_volatile(const long long* p) {
  return *(const volatile long long*)p;
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Release/acquire fence at GPU scope. A relaxed write after it is a release
// of everything before it; a relaxed read before it is an acquire for
// everything after it. It does not order a write before a later read of
// another location, so the two places that need that (rank writes before the
// state-word check, state change before reading contributions) keep the
// sequentially consistent __threadfence().
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void atomic_add_ll(long long* p, long long v) {
  atomicAdd((unsigned long long*)p, (unsigned long long)v);
}
__device__ __forceinline__ long long atomic_add_ll_old(long long* p, long long v) {
  return (long long)atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

// ---------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------

// FP64 ranks; contributions in 64-bit fixed point (scale 2^60, see
// contrib_of), summed exactly with integer adds.
struct P64 {
  using val = double;
  using contrib = long long;
  using acc = long long;
  static __device__ __forceinline__ acc zero() { return 0ll; }
  static __device__ __forceinline__ acc from(contrib x) { return x; }
  static __device__ __forceinline__ acc add(acc a, acc b) { return a + b; }
  static __device__ __forceinline__ double total(acc a) { return __ll2double_rn(a) * kInvFix; }
  static __device__ __forceinline__ double value(contrib c) { return __ll2double_rn(c) * kInvFix; }
  static __device__ __forceinline__ acc shfl_up(acc a, int d) { return __shfl_up_sync(kFull, a, d); }
  static __device__ __forceinline__ val load(const val* p) { return __ldcg(p); }
  static __device__ __forceinline__ contrib load_c(const contrib* p) { return __ldcg(p); }
  static __device__ __forceinline__ acc shfl_xor(acc a, int d) { return __shfl_xor_sync(kFull, a, d); }
  // per-vertex record: {rank, x} | {in-row, out-degree | flags << 32}
  static __device__ __forceinline__ void load_rec(const VRec* p, val& r, val& x, long long& ioff,
                                                  int& ideg, int& od, unsigned& fl) {
    const longlong2 u = __ldcg(reinterpret_cast<const longlong2*>(p));
    const longlong2 w = __ldcg(reinterpret_cast<const longlong2*>(p) + 1);
    r = __longlong_as_double(u.x);
    x = __longlong_as_double(u.y);
    ioff = (long long)((unsigned long long)w.x >> 25);
    ideg = (int)(w.x & 0x1ffffffll);
    od = (int)(w.y & 0xffffffffll);
    fl = (unsigned)((unsigned long long)w.y >> 32);
  }
  static __device__ __forceinline__ void init_rec(VRec* p, val r, long long ioff, int ideg, int od) {
    longlong2 u, w;
    u.x = __double_as_longlong(r);
    u.y = __double_as_longlong(r);
    w.x = (long long)(((unsigned long long)ioff << 25) | (unsigned long long)ideg);
    w.y = (long long)(unsigned)od;
    reinterpret_cast<longlong2*>(p)[0] = u;
    reinterpret_cast<longlong2*>(p)[1] = w;
  }
  static __device__ __forceinline__ void store_rx(VRec* p, val r, val x) {
    longlong2 u;
    u.x = __double_as_longlong(r);
    u.y = __double_as_longlong(x);
    *reinterpret_cast<longlong2*>(p) = u;
  }
  static __device__ __forceinline__ void set_fresh(VRec* p) { reinterpret_cast<unsigned*>(p)[7] = 1u; }
  static __device__ __forceinline__ val rec_rank(const VRec* p) {
    return __longlong_as_double(*reinterpret_cast<const long long*>(p));
  }
  // heavy-gather jobs: partial sums meet in one 64-bit word (exact integer adds)
  static __device__ __forceinline__ void job_add(unsigned long long* p, acc x) {
    atomicAdd(p, (unsigned long long)x);
  }
  static __device__ __forceinline__ double job_total(unsigned long long bits) {
    return __ll2double_rn((long long)bits) * kInvFix;
  }
  static constexpr bool relative = false;
  // the worklist epilogue solves the self-loop term of Eq. 1 in closed form
  static constexpr bool closed_form = true;
};

// FP32 with compensated summation: every addition is an error-free TwoSum
// (Knuth); the rounding errors are carried in a second float.
struct CompF {
  float s, c;
};
struct P32 {
  using val = float;
  using contrib = float;
  using acc = CompF;
  static __device__ __forceinline__ acc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ acc from(contrib x) { return {x, 0.f}; }
  static __device__ __forceinline__ acc add(acc a, acc b) {
    const float s = __fadd_rn(a.s, b.s);
    const float bp = __fsub_rn(s, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(b.s, bp));
    return {s, __fadd_rn(__fadd_rn(a.c, b.c), err)};
  }
  static __device__ __forceinline__ double total(acc a) { return (double)a.s + (double)a.c; }
  static __device__ __forceinline__ double value(contrib c) { return (double)c; }
  static __device__ __forceinline__ acc shfl_up(acc a, int d) {
    return {__shfl_up_sync(kFull, a.s, d), __shfl_up_sync(kFull, a.c, d)};
  }
  static __device__ __forceinline__ val load(const val* p) { return __ldcg(p); }
  static __device__ __forceinline__ contrib load_c(const contrib* p) { return __ldcg(p); }
  // per-vertex record: {rank, x, out-degree, flags} | {in-row, unused}
  static __device__ __forceinline__ void load_rec(const VRec* p, val& r, val& x, long long& ioff,
                                                  int& ideg, int& od, unsigned& fl) {
    const uint4 u = __ldcg(reinterpret_cast<const uint4*>(p));
    const unsigned long long in = __ldcg(reinterpret_cast<const unsigned long long*>(p) + 2);
    r = __uint_as_float(u.x);
    x = __uint_as_float(u.y);
    od = (int)u.z;
    fl = u.w;
    ioff = (long long)(in >> 25);
    ideg = (int)(in & 0x1ffffffull);
  }
  static __device__ __forceinline__ void init_rec(VRec* p, val r, long long ioff, int ideg, int od) {
    reinterpret_cast<uint4*>(p)[0] = make_uint4(__float_as_uint(r), __float_as_uint(r), (unsigned)od, 0u);
    reinterpret_cast<unsigned long long*>(p)[2] = ((unsigned long long)ioff << 25) | (unsigned long long)ideg;
    reinterpret_cast<unsigned long long*>(p)[3] = 0ull;
  }
  static __device__ __forceinline__ void store_rx(VRec* p, val r, val x) {
    *reinterpret_cast<uint2*>(p) = make_uint2(__float_as_uint(r), __float_as_uint(x));
  }
  static __device__ __forceinline__ void set_fresh(VRec* p) { reinterpret_cast<unsigned*>(p)[3] = 1u; }
  static __device__ __forceinline__ val rec_rank(const VRec* p) {
    return __uint_as_float(*reinterpret_cast<const unsigned*>(p));
  }
  static __device__ __forceinline__ acc shfl_xor(acc a, int d) {
    return {__shfl_xor_sync(kFull, a.s, d), __shfl_xor_sync(kFull, a.c, d)};
  }
  // heavy-gather jobs: partial sums meet in one FP64 word
  static __device__ __forceinline__ void job_add(unsigned long long* p, acc x) {
    atomicAdd(reinterpret_cast<double*>(p), total(x));
  }
  static __device__ __forceinline__ double job_total(unsigned long long bits) {
    return __longlong_as_double((long long)bits);
  }
  static constexpr bool relative = true;
  // Eq. 1 as printed, the vertex's current rank in its self-loop term: FP32
  // rounding jitter under a relative, one-ulp frontier floor needs that damping
  static constexpr bool closed_form = false;
};

// ---------------------------------------------------------------------------
// Kernel arguments
// ---------------------------------------------------------------------------

// Frontier threshold of a vertex with new rank r: tau_f absolute (FP64), or
// tau_f relative to r but at least one unit in the last place of r (FP32: a
// threshold below one ulp would expand on every rounding jitter).
template <class P>
__device__ __forceinline__ double frontier_thr(double tol_f, typename P::val r) {
  if (!P::relative) return tol_f;
  const float fr = fabsf((float)r);
  const float ulp = __int_as_float(__float_as_int(fr) & 0x7f800000) * 1.1920928955078125e-7f;
  return fmax(tol_f * (double)fr, (double)ulp);
}

template <class P>
struct Args {
  int32_t n;
  const RowDesc* __restrict__ in_rows;
  const int32_t* __restrict__ in_edges;
  const RowDesc* __restrict__ out_rows;
  const int32_t* __restrict__ out_edges;
  typename P::val* R;
  typename P::contrib* C;
  VRec* rec;
  uint32_t* state;
  int32_t* queue;
  unsigned long long qmask;
  DfCtl* ctl;
  // marking items
  const int32_t* mark_src;
  const long long* mark_choff;  // exclusive scan of marking chunks per source
  long long n_mark_src;
  const int32_t* mark_dst;
  long long n_mark_dst;
  // round mode
  uint32_t* va_bits;
  uint32_t* rc_bits;
  int32_t* alist;
  unsigned long long* pass_ctr;
  uint32_t* item_done;
  int max_iter;
  // worklist: token ring and heavy-gather jobs
  unsigned long long* tokens;
  unsigned long long tmask;
  int32_t* job_ring;
  int32_t* job_v;
  int32_t* job_rem;
  unsigned long long* job_sum;
  unsigned jmask;
  // a set of graphs: vertex offsets, per-graph completion times
  const int32_t* part_off;
  int nparts;
  unsigned long long* part_done;
  // numerics
  double alpha, base, tol, tol_f;
  int teleport;
  unsigned long long timeout_ns;
  int mark_only;
  int gather_split;  // in-edges per gather token (longer in-rows are split)
  int mark_split;    // out-edges per mark token (longer out-rows are split)
  // simulated faults (Sec. 5.1.6): per-vertex delay probability as a 64-bit
  // threshold, delay length, crashing warps = those whose slot in a seeded
  // permutation of the launch's warps is below fault_crash_warps
  unsigned long long fault_seed;
  unsigned long long fault_delay_thr;
  unsigned long long fault_delay_ns;
  unsigned long long fault_perm_a, fault_perm_b;
  unsigned long long fault_warps;
  int fault_crash_warps;
  // helping (worklist): per-warp hold records, kHoldWords 64-bit words each
  unsigned long long* hold;
  int helping;
  // jacobi: in-rows longer than gather_split, registered per iteration and
  // summed in gather_split-edge chunks by every warp (jh_cap slots)
  int32_t* jh_v;
  int32_t* jh_rem;
  unsigned long long* jh_sum;
  long long* jh_off;
  long long jh_cap;
};

// Per-warp statistics: counters in shared memory that lane 0 updates with
// warp totals (so they hold no registers), and each lane's largest change.
enum {
  kStEdges, kStExpansions, kStMarked, kStPushes, kStAffected,  // flushed by every kernel
  kStBatches, kStPhase0, kStTokens = kStPhase0 + 5, kStJobs,   // worklist only
  kStProcessed, kStClock, kStCount
};
struct WarpStats {
  unsigned long long* c;  // kStCount counters of this warp (shared memory)
  double max_change;
};

// Points st at this warp's counters and clears them (warp-uniform call).
__device__ __forceinline__ void stats_init(WarpStats& st, unsigned long long* c, int lane) {
  st.c = c;
  st.max_change = 0.0;
  if (lane < kStCount) c[lane] = 0ull;
  __syncwarp();
}

// Adds the number of lanes with `pred` to counter k (warp-uniform call).
__device__ __forceinline__ void stats_count(WarpStats& st, int k, bool pred, int lane) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if (lane == 0 && b) st.c[k] += (unsigned long long)__popc(b);
}

// (1 - alpha) / n of the graph that holds v (Eq. 1 per graph of a set).
template <class P>
__device__ __forceinline__ double base_of(const Args<P>& a, int v) {
  if (a.nparts <= 1) return a.base;
  const int p = part_of(a.part_off, a.nparts, v);
  return (1.0 - a.alpha) / (double)(__ldg(a.part_off + p + 1) - __ldg(a.part_off + p));
}

template <class P>
__device__ __forceinline__ bool timed_out(const Args<P>& a) {
  return gtime() - a.ctl->t_start > a.timeout_ns;
}

// ---------------------------------------------------------------------------
// Simulated thread delays and crash-stops (Sec. 5.1.6)
// ---------------------------------------------------------------------------

// SplitMix64 finaliser (Steele, Lea, Flood 2014): a counter-based hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

constexpr unsigned long long kCrashHorizon = 64;  // a crashing warp stops within its first 64 batches

__device__ __forceinline__ unsigned long long fault_warp_id() {
  return (unsigned long long)blockIdx.x * kWPB + (threadIdx.x >> 5);
}

// True when this warp is one of the crashing ones and its batch number k is
// its crash point (a crash-stop: the caller returns at once, leaving any
// bookkeeping undone).
template <class P>
__device__ __forceinline__ bool fault_crash(const Args<P>& a, unsigned long long k) {
  if (a.fault_crash_warps == 0) return false;
  const unsigned long long gid = fault_warp_id();
  const unsigned long long slot = (gid * a.fault_perm_a + a.fault_perm_b) % a.fault_warps;
  return slot < (unsigned long long)a.fault_crash_warps &&
         k == mix64(a.fault_seed ^ mix64(gid)) % kCrashHorizon;
}

// Thread delay after a warp's batch number k (warp-uniform call; has_vertex:
// this lane recomputed a vertex in it): with probability fault_delay_prob per
// vertex the warp sleeps fault_delay_ns, in a bounded loop that also ends at
// the time budget.
template <class P>
__device__ __forceinline__ void fault_delay(const Args<P>& a, unsigned long long k, bool has_vertex,
                                           int lane) {
  if (a.fault_delay_thr == 0ull) return;
  const unsigned long long h = mix64(a.fault_seed ^ mix64(fault_warp_id()) ^ 0x6a09e667f3bcc909ull);
  const bool hit = has_vertex && mix64(h + (k << 5) + (unsigned long long)lane) < a.fault_delay_thr;
  if (!__any_sync(kFull, hit)) return;
  const unsigned long long t0 = gtime();
  while (gtime() - t0 < a.fault_delay_ns) {
    if (gtime() - a.ctl->t_start > a.timeout_ns) break;
    __nanosleep(100000);
  }
}

template <class P>
__device__ void stop_with(const Args<P>& a, unsigned status) {
  atomicCAS(&a.ctl->status, 0u, status);
  atomicExch(&a.ctl->abort, 1u);
}

// Row descriptor through the read-only path (rows do not change during a kernel).
__device__ __forceinline__ RowDesc load_row(const RowDesc* p) {
  const longlong2 x = __ldg(reinterpret_cast<const longlong2*>(p));
  RowDesc r;
  r.off = x.x;
  r.deg = (int)(x.y & 0xffffffffll);
  r.cap = (int)(x.y >> 32);
  return r;
}

// Last index j in [0, 32) with s_excl[j] <= e (s_excl nondecreasing, s_excl[0] = 0).
__device__ __forceinline__ int owner_of(const int* s_excl, int e) {
  int lo = 0, hi = 32;
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const int mid = (lo + hi) >> 1;
    if (s_excl[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// 32-edge chunks whose loads are in flight at once per warp. Measured on
// R-MAT scale 24: 2 chunks beat 4 (about 131 vs 147 ms per update), and 6 or
// 8 were slower still. The random contribution reads oversubscribe the
// memory system well before per-warp concurrency runs out.
constexpr int kUnroll = 2;

// Loads the ids of kUnroll 32-edge chunks of a warp's concatenated edge list,
// starting at edge `base`: lane i takes edges base + 32k + i. owner[k] is the
// lane whose row holds the edge (-1 past the end).
__device__ __forceinline__ void load_chunk_ids(const int32_t* __restrict__ edges, const int* s_excl,
                                               const long long* s_off, int base, int total, int lane,
                                               int (&owner)[kUnroll], int (&id)[kUnroll]) {
#pragma unroll
  for (int k = 0; k < kUnroll; ++k) {
    const int e = base + k * 32 + lane;
    owner[k] = -1;
    id[k] = 0;
    if (e < total) {
      const int o = owner_of(s_excl, e);
      owner[k] = o;
      id[k] = __ldg(edges + s_off[o] + (e - s_excl[o]));
    }
  }
}

// Warp-cooperative edge-balanced gather: lane i owns vertex v_i (or -1).
// Returns sum_{u in in(v_i)} C[u] in lane i. The in-edges of the 32 vertices
// are walked as one list, kUnroll chunks of 32 at a time. The loop is
// software-pipelined: the ids of the next kUnroll chunks are loaded while the
// contributions of the current ones are in flight, so each step waits for one
// memory round trip, not two. Each chunk is reduced by a segmented warp scan
// whose segment tails add into s_acc[owner].
template <class P>
__device__ typename P::acc gather_row(const Args<P>& a, int deg, long long off, int lane, int* s_excl,
                                      long long* s_off, typename P::acc* s_acc, WarpStats& st) {
  int incl = deg;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  s_excl[lane] = incl - deg;
  s_off[lane] = off;
  s_acc[lane] = P::zero();
  __syncwarp();
  int owner[kUnroll], uid[kUnroll];
  if (total > 0) load_chunk_ids(a.in_edges, s_excl, s_off, 0, total, lane, owner, uid);
  for (int base = 0; base < total; base += 32 * kUnroll) {
    typename P::contrib xv[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k)
      xv[k] = owner[k] >= 0 ? P::load_c(a.C + uid[k]) : (typename P::contrib)0;
    int owner_n[kUnroll], uid_n[kUnroll];
    load_chunk_ids(a.in_edges, s_excl, s_off, base + 32 * kUnroll, total, lane, owner_n, uid_n);
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      if (base + k * 32 >= total) break;  // warp-uniform
      typename P::acc x = P::from(xv[k]);
      const int key = owner[k] >= 0 ? owner[k] : 32 + lane;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const typename P::acc y = P::shfl_up(x, d);
        const int k2 = __shfl_up_sync(kFull, key, d);
        if (lane >= d && k2 == key) x = P::add(x, y);
      }
      const int knext = __shfl_down_sync(kFull, key, 1);
      if (owner[k] >= 0 && (lane == 31 || knext != key)) s_acc[key] = P::add(s_acc[key], x);
      __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      owner[k] = owner_n[k];
      uid[k] = uid_n[k];
    }
  }
  if (lane == 0) st.c[kStEdges] += (unsigned long long)total;
  return s_acc[lane];
}

// gather_row over the in-row of v (nothing when v < 0).
template <class P>
__device__ __forceinline__ typename P::acc gather(const Args<P>& a, int v, int lane, int* s_excl,
                                                  long long* s_off, typename P::acc* s_acc,
                                                  WarpStats& st) {
  RowDesc r;
  r.off = 0;
  r.deg = 0;
  if (v >= 0) r = load_row(a.in_rows + v);
  return gather_row(a, r.deg, r.off, lane, s_excl, s_off, s_acc, st);
}

// Per-warp buffer of queue insertions in shared memory, flushed to the ring
// once per batch (or when full), so that a batch pays one fence and one
// round of counter atomics for all its insertions.
constexpr int kPushCap = 256;
struct PushBuf {
  int* items;
  int* cnt;   // items buffered
  int* nnew;  // of which newly queued (they add to `pending`)
  int* owed;  // completions not yet subtracted from `pending`
};

// Applies this warp's deferred completions to `pending` (lane 0). Deferring a
// decrement only over-counts, so it is always safe; an idle warp settles its
// debt before it tests for termination.
template <class P>
__device__ void settle_owed(const Args<P>& a, PushBuf pb, int lane) {
  __syncwarp();
  if (lane == 0 && *pb.owed) {
    atomic_add_ll(&a.ctl->pending.v, -(long long)*pb.owed);
    *pb.owed = 0;
  }
  __syncwarp();
}

template <class P>
__device__ bool buf_flush(const Args<P>& a, PushBuf pb, int lane, WarpStats& st) {
  __syncwarp();
  const int cnt = *pb.cnt;
  if (cnt == 0) return true;
  const int nnew = *pb.nnew;
  unsigned long long base = 0;
  if (lane == 0) {
    // `pending` grows before any of these items becomes visible in the ring,
    // so it cannot reach zero while they are outstanding; the warp's deferred
    // completions ride on the same atomic
    const long long delta = (long long)nnew - (long long)*pb.owed;
    *pb.owed = 0;
    if (delta) atomic_add_ll(&a.ctl->pending.v, delta);
    fence_acq_rel();
    base = atomicAdd(&a.ctl->tail.v, (unsigned long long)cnt);
    st.c[kStPushes] += (unsigned long long)cnt;
  }
  base = __shfl_sync(kFull, base, 0);
  bool ok = true;
  for (int i = lane; i < cnt; i += 32) {
    int* slot = a.queue + ((base + (unsigned long long)i) & a.qmask);
    unsigned spins = 0;
    while (ld_volatile(slot) != -1) {  // slot still held by a slow consumer
      if ((++spins & 255u) == 0 && timed_out(a)) {
        stop_with(a, DFPR_ETIMEOUT);
        ok = false;
        break;
      }
      __nanosleep(64);
    }
    if (!ok) break;
    *(volatile int*)slot = pb.items[i];
  }
  __syncwarp();
  if (lane == 0) {
    atomic_add_ll(&a.ctl->avail.v, cnt);  // consumers wait on the slots themselves
    *pb.cnt = 0;
    *pb.nnew = 0;
  }
  __syncwarp();
  return __all_sync(kFull, ok);
}

// Buffers t for every lane with need (warp-uniform call).
template <class P>
__device__ void buf_push(const Args<P>& a, PushBuf pb, int t, bool need, bool is_new, int lane,
                         WarpStats& st) {
  const unsigned b = __ballot_sync(kFull, need);
  if (!b) return;
  const int k = __popc(b);
  if (*pb.cnt + k > kPushCap) buf_flush(a, pb, lane, st);
  const int c = *pb.cnt;
  if (need) pb.items[c + __popc(b & lanemask_lt())] = t;
  __syncwarp();
  if (lane == 0) {
    *pb.cnt = c + k;
    if (is_new) *pb.nnew += k;
  }
  __syncwarp();
}

// Marks t (lanes with valid): sets its queued bit and buffers it when it was
// idle. A plain load first skips the atomic when the bit is already set; that
// is safe because the caller fenced its rank writes before marking, and a
// worker clears the bit (and fences) before reading contributions.
template <class P>
__device__ __forceinline__ bool mark_one(const Args<P>& a, int t, bool valid, unsigned word) {
  if (!valid) return false;
  const unsigned sh = (unsigned)(t & 15) * 2u;
  if ((word >> sh) & 1u) return false;
  const unsigned old = atomicOr(a.state + (t >> 4), 1u << sh);
  return ((old >> sh) & 3u) == 0u;
}

// Tokens: bit 63..62 kind, 61..31 a, 30..0 b. Kind 0: gather chunk b of job
// slot a. Kind 1: mark chunk b of vertex a's out-row.
// Default in-edges per gather token and out-edges per mark token (longer
// rows are split; dfpr_params.gather_split / mark_split override them, and
// dfpr_autotune picks them by timing). Measured on R-MAT scale 24: 4096 /
// 8192 took 107 ms per update, 2048 / 2048 115 ms, 1024 / 1024 182 ms (token
// and job overhead), and 16384 / 16384 138 ms (too few pieces to spread a
// hub over the GPU).
constexpr int kGatherChunk = 4096;
constexpr int kMarkSplit = 8192;
constexpr unsigned long long kNoToken = ~0ull;

__device__ __forceinline__ unsigned long long make_token(unsigned kind, unsigned x, unsigned y) {
  return ((unsigned long long)kind << 62) | ((unsigned long long)x << 31) | (unsigned long long)y;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// Every lane publishes `cnt` tokens make_token(kind, x, k), k < cnt (warp-uniform call).
// `pending` grows first, so the iteration cannot end while they are outstanding.
template <class P>
__device__ void push_tokens(const Args<P>& a, int cnt, unsigned kind, unsigned x, int lane,
                            WarpStats& st, long long* open) {
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) {
    atomic_add_ll(open, total);
    fence_acq_rel();
    base = atomicAdd(&a.ctl->ttail.v, (unsigned long long)total);
  }
  base = __shfl_sync(kFull, base, 0);
  bool ok = true;
  for (int k = 0; k < cnt && ok; ++k) {
    unsigned long long* slot = a.tokens + ((base + (unsigned long long)(incl - cnt + k)) & a.tmask);
    unsigned spins = 0;
    while (ld_volatile(slot) != kNoToken) {  // slot still held by a slow consumer
      if ((++spins & 255u) == 0 && timed_out(a)) {
        stop_with(a, DFPR_ETIMEOUT);
        ok = false;
        break;
      }
      __nanosleep(64);
    }
    if (ok) *(volatile unsigned long long*)slot = make_token(kind, x, (unsigned)k);
  }
  fence_acq_rel();
  __syncwarp();
  if (lane == 0) atomic_add_ll(&a.ctl->tavail.v, total);
}

// Claims one token (lane 0; result broadcast), or returns kNoToken.
template <class P>
__device__ unsigned long long pop_token(const Args<P>& a, int lane) {
  unsigned long long tok = kNoToken;
  if (lane == 0 && ld_volatile(&a.ctl->tavail.v) > 0) {
    if (atomic_add_ll_old(&a.ctl->tavail.v, -1) > 0) {
      const unsigned long long pos = atomicAdd(&a.ctl->thead.v, 1ull);
      unsigned long long* slot = a.tokens + (pos & a.tmask);
      unsigned spins = 0;
      while ((tok = ld_volatile(slot)) == kNoToken) {  // producer between claim and write
        if ((++spins & 255u) == 0 && timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          break;
        }
        __nanosleep(32);
      }
      if (tok != kNoToken) *(volatile unsigned long long*)slot = kNoToken;
    } else {
      atomic_add_ll(&a.ctl->tavail.v, 1);
    }
  }
  return __shfl_sync(kFull, tok, 0);
}

// Takes a free heavy-gather job slot (per lane), or -1 when none is free.
template <class P>
__device__ int alloc_job(const Args<P>& a) {
  if (ld_volatile(&a.ctl->favail.v) <= 0) return -1;
  if (atomic_add_ll_old(&a.ctl->favail.v, -1) <= 0) {
    atomic_add_ll(&a.ctl->favail.v, 1);
    return -1;
  }
  const unsigned long long pos = atomicAdd(&a.ctl->fhead.v, 1ull);
  int* slot = a.job_ring + (pos & a.jmask);
  int id;
  unsigned spins = 0;
  while ((id = ld_volatile(slot)) < 0) {
    if ((++spins & 255u) == 0 && timed_out(a)) {
      stop_with(a, DFPR_ETIMEOUT);
      return -1;
    }
    __nanosleep(32);
  }
  *(volatile int*)slot = -1;
  return id;
}

template <class P>
__device__ void free_job(const Args<P>& a, int id) {
  const unsigned long long pos = atomicAdd(&a.ctl->ftail.v, 1ull);
  int* slot = a.job_ring + (pos & a.jmask);
  unsigned spins = 0;
  while (ld_volatile(slot) != -1) {
    if ((++spins & 255u) == 0 && timed_out(a)) {
      stop_with(a, DFPR_ETIMEOUT);
      return;
    }
    __nanosleep(32);
  }
  *(volatile int*)slot = id;
  fence_acq_rel();
  atomic_add_ll(&a.ctl->favail.v, 1);
}

// Marks the out-neighbours of every lane's vertex v (with od > 0 out-edges at
// oo). Out-rows longer than a.mark_split become mark tokens that any warp takes;
// the rest are walked edge-balanced, kUnroll chunks in flight.
template <class P>
__device__ void expand_rows(const Args<P>& a, int v, int od, long long oo, int lane, int* s_excl,
                            long long* s_off, PushBuf pb, WarpStats& st) {
  const bool split = od > a.mark_split;
  push_tokens(a, split ? (od + a.mark_split - 1) / a.mark_split : 0, 1u, (unsigned)max(v, 0), lane, st,
              &a.ctl->pending.v);
  if (split) od = 0;
  int incl = od;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  if (total == 0) return;
  __syncwarp();
  s_excl[lane] = incl - od;
  s_off[lane] = oo;
  __syncwarp();
  int own[kUnroll], t[kUnroll];
  load_chunk_ids(a.out_edges, s_excl, s_off, 0, total, lane, own, t);
  for (int base = 0; base < total; base += 32 * kUnroll) {
    unsigned wv[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) wv[k] = own[k] >= 0 ? ld_volatile(a.state + (t[k] >> 4)) : 0u;
    int own_n[kUnroll], t_n[kUnroll];
    load_chunk_ids(a.out_edges, s_excl, s_off, base + 32 * kUnroll, total, lane, own_n, t_n);
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      if (base + k * 32 >= total) break;  // warp-uniform
      // with the closed form, the row owner's own self-loop is not marked:
      // its rank is exact in itself
      const int owner_v = __shfl_sync(kFull, v, own[k] >= 0 ? own[k] : 0);
      const bool need = mark_one(a, t[k], own[k] >= 0 && !(P::closed_form && t[k] == owner_v), wv[k]);
      buf_push(a, pb, t[k], need, true, lane, st);
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      own[k] = own_n[k];
      t[k] = t_n[k];
    }
  }
  if (lane == 0) st.c[kStMarked] += (unsigned long long)total;
}

// Marking item: a chunk of a source's out-row, or up to 32 deletion targets.
// For the DF approach (Sec. 4.1) the affected set is out_{t-1}(u) union
// out_t(u) = out_t(u) plus the targets of u's deleted edges.
template <class P, class MarkFn>
__device__ void do_mark_item(const Args<P>& a, long long item, int lane, WarpStats& st, MarkFn mark) {
  const long long n_src_items = (long long)a.ctl->n_src_items;
  if (item < n_src_items) {
    long long lo = 0, hi = a.n_mark_src;  // last s with choff[s] <= item
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (a.mark_choff[mid] <= item) lo = mid; else hi = mid;
    }
    const int u = a.mark_src[lo];
    const long long chunk = item - a.mark_choff[lo];
    const RowDesc r = load_row(a.out_rows + u);
    const long long beg = chunk * kMarkChunk;
    const long long end = min((long long)r.deg, beg + kMarkChunk);
    for (long long e0 = beg; e0 < end; e0 += 32) {
      const long long e = e0 + lane;
      const bool valid = e < end;
      const int t = valid ? __ldg(a.out_edges + r.off + e) : 0;
      mark(t, valid);
    }
    if (lane == 0) st.c[kStMarked] += (unsigned long long)max(0ll, end - beg);
  } else {
    const long long j = (item - n_src_items) * 32 + lane;
    const long long n_mark_dst = a.ctl->n_mark_dst;
    const bool valid = j < n_mark_dst;
    const int t = valid ? a.mark_dst[j] : 0;
    mark(t, valid);
    if (lane == 0) st.c[kStMarked] += (unsigned long long)min(32ll, n_mark_dst - (item - n_src_items) * 32);
  }
}

template <class P>
__device__ void flush_stats(const Args<P>& a, WarpStats& st, int lane) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1)
    st.max_change = fmax(st.max_change, __shfl_down_sync(kFull, st.max_change, d));
  __syncwarp();
  if (lane == 0) {
    DfCtl* c = a.ctl;
    const unsigned long long* k = st.c;
    if (k[kStEdges]) atomicAdd(&c->edges, k[kStEdges]);
    if (k[kStExpansions]) atomicAdd(&c->expansions, k[kStExpansions]);
    if (k[kStMarked]) atomicAdd(&c->edges_marked, k[kStMarked]);
    if (k[kStPushes]) atomicAdd(&c->pushes, k[kStPushes]);
    if (k[kStAffected]) atomicAdd(&c->affected, k[kStAffected]);
    if (st.max_change > 0) atomicMax(&c->max_change_bits, (unsigned long long)__double_as_longlong(st.max_change));
  }
}

// Eq. 1 for a recomputed vertex v, from its gathered sum.
template <class P>
__device__ __forceinline__ typename P::val finish_rank(const Args<P>& a, typename P::acc acc,
                                                       double dangling, int v) {
  double s = P::total(acc);
  if (a.teleport) s += dangling / (double)a.n;
  return (typename P::val)(base_of(a, v) + a.alpha * s);
}

// Records, per graph of a set, when a warp last finished a vertex of it
// (warp-uniform call; one atomic per distinct graph in the warp).
template <class P>
__device__ __forceinline__ void note_done(const Args<P>& a, int v, int lane) {
  if (a.nparts <= 1) return;
  const int p = v >= 0 ? part_of(a.part_off, a.nparts, v) : -1;
  const unsigned grp = __match_any_sync(kFull, p);
  if (p >= 0 && __ffs(grp) - 1 == lane) atomicMax(a.part_done + p, gtime());
}

// ---------------------------------------------------------------------------
// Worklist schedule
// ---------------------------------------------------------------------------

constexpr double kDriftFactor = 10.0;

// Eq. 1 epilogue of one recomputed vertex v on the per-vertex record. Every
// vertex of the worklist schedule has a self-loop (dead ends are removed that
// way, Sec. 5.1.3), so its own rank is one of its inputs: r = b + alpha *
// (S + r / |out(v)|), S the sum over its other in-edges.
//  - FP64 (P::closed_form) solves that term: r = (b + alpha * S) /
//    (1 - alpha / |out(v)|), the same fixed point as Eq. 1. The recomputation
//    is exact in v's own rank, so v never revisits itself because its own rank
//    moved: its expansion marks its other out-neighbours only, and it is not
//    queued again for its own change. The sums are exact integers and the
//    frontier threshold is absolute, so rounding cannot move a rank by it.
//  - FP32 evaluates Eq. 1 as printed, with v's current rank in the self term:
//    a vertex whose rank moved marks itself (its self-loop) on expansion, and
//    queues itself again while its own change is above tau. Under the relative
//    tolerance with its one-ulp floor, the closed form's undamped rounding
//    jitter let neighbours flip each other by an ulp or two for ever.
// sum is the gather over the whole in-row, the self-loop included; the closed
// form subtracts its term, the stored contribution of r_old. The rank at the
// last expansion (initialised to the rank at the call's start) decides
// whether v marks its out-neighbours. Writes the record's rank and x, the
// recomputed flag, and C.
template <class P>
__device__ __forceinline__ void vertex_epilogue_rec(const Args<P>& a, int v, double sum,
                                                    typename P::val r_old, typename P::val x0,
                                                    unsigned fl, int od, double dangling,
                                                    bool& expand, bool& requeue, bool& fresh,
                                                    WarpStats& st) {
  (void)dangling;  // the worklist schedule has no dead ends
  typename P::val r;
  if constexpr (P::closed_form) {
    const double others = sum - P::value(contrib_of(r_old, od));
    const double r_exact = (base_of(a, v) + a.alpha * others) / (1.0 - a.alpha / (double)od);
    // a rank is at most 1 at the fixed point; stale inputs of a vertex with
    // few out-edges can push the closed form above it for a moment, and the
    // fixed-point contributions must stay bounded
    r = (typename P::val)fmin(fmax(r_exact, 0.0), 1.0);
  } else {
    r = (typename P::val)(base_of(a, v) + a.alpha * sum);
  }
  fresh = (fl & 1u) == 0u;
  const double dr = fabs((double)r - (double)r_old);
  a.C[v] = contrib_of(r, od);
  const double thr_f = frontier_thr<P>(a.tol_f, r);
  const double drift = fabs((double)r - (double)x0);
  expand = P::relative ? drift > thr_f : (dr > thr_f || drift > kDriftFactor * thr_f);
  requeue = !P::closed_form && dr > (P::relative ? a.tol * fabs((double)r) : a.tol);
  P::store_rx(a.rec + v, r, expand ? r : x0);
  if (fresh) P::set_fresh(a.rec + v);
  st.max_change = fmax(st.max_change, dr);
}

// After the epilogue of lane-local vertices: marks out-neighbours of expanding
// ones, flags the vertices to requeue (FP32: own change above tau), and moves
// each vertex from running to idle (or back to queued when it was flagged
// meanwhile). Returns the number of vertices that left the system (their
// `pending` units are owed).
template <class P>
__device__ int finish_vertices(const Args<P>& a, int v, bool expand, bool requeue, RowDesc orow,
                               int lane, int* s_excl, long long* s_off, PushBuf pb, WarpStats& st) {
  __threadfence();  // new ranks visible before neighbours are queued
  expand_rows(a, v, expand ? orow.deg : 0, orow.off, lane, s_excl, s_off, pb, st);
  if (requeue && !expand) {  // flags itself so that the finish re-queues it
    const unsigned sh = (unsigned)(v & 15) * 2u;
    atomicOr(a.state + (v >> 4), 1u << sh);
  }
  bool repush = false;
  if (v >= 0) {
    const unsigned sh = (unsigned)(v & 15) * 2u;
    const unsigned old = atomicAnd(a.state + (v >> 4), ~(2u << sh));
    repush = ((old >> sh) & 1u) != 0u;
  }
  buf_push(a, pb, v, repush, false, lane, st);
  buf_flush(a, pb, lane, st);
  return __popc(__ballot_sync(kFull, v >= 0 && !repush));
}

// Gather token: sums one chunk of a heavy vertex's in-row into its job; the
// warp that sums the last chunk finishes the vertex.
// Sums chunk `chunk` of the in-row of job `slot`'s vertex into the job
// (exact integer adds in FP64 mode). Returns, warp-uniform, whether this warp
// summed the last chunk; *vout receives the vertex.
template <class P>
__device__ bool sum_gather_token(const Args<P>& a, unsigned slot, unsigned chunk, int lane,
                                 WarpStats& st, int* vout) {
  fence_acq_rel();  // the job record was published before the token
  const int v = ld_volatile(a.job_v + slot);
  const RowDesc row = load_row(a.in_rows + v);
  const long long beg = (long long)chunk * a.gather_split;
  const long long end = min((long long)row.deg, beg + a.gather_split);
  typename P::acc acc = P::zero();
  for (long long e0 = beg; e0 < end; e0 += 32 * kUnroll) {
    typename P::contrib xv[kUnroll];
    int uid[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const long long e = e0 + k * 32 + lane;
      uid[k] = e < end ? __ldg(a.in_edges + row.off + e) : -1;
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) xv[k] = uid[k] >= 0 ? P::load_c(a.C + uid[k]) : (typename P::contrib)0;
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) acc = P::add(acc, P::from(xv[k]));
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc = P::add(acc, P::shfl_xor(acc, d));
  int last = 0;
  if (lane == 0) {
    P::job_add(a.job_sum + slot, acc);
    fence_acq_rel();
    last = atomicSub(a.job_rem + slot, 1) == 1;
    st.c[kStEdges] += (unsigned long long)max(0ll, end - beg);
  }
  *vout = v;
  return __shfl_sync(kFull, last, 0) != 0;
}

template <class P>
__device__ int run_gather_token(const Args<P>& a, unsigned slot, unsigned chunk, int lane,
                                int* s_excl, long long* s_off, PushBuf pb, WarpStats& st) {
  int v = -1;
  if (!sum_gather_token(a, slot, chunk, lane, st, &v)) return 0;
  // finish the heavy vertex (lane 0 owns it)
  fence_acq_rel();
  const int vv = lane == 0 ? v : -1;
  bool expand = false, requeue = false, fresh = false;
  RowDesc orow;
  orow.off = 0;
  orow.deg = 0;
  if (vv >= 0) {
    const double sum = P::job_total(ld_volatile(a.job_sum + slot));
    typename P::val r_old, x_prev;
    long long ioff;
    int ideg, od;
    unsigned fl;
    P::load_rec(a.rec + vv, r_old, x_prev, ioff, ideg, od, fl);
    const double dangling = a.teleport ? a.ctl->dsum : 0.0;
    vertex_epilogue_rec(a, vv, sum, r_old, x_prev, fl, od, dangling, expand, requeue, fresh, st);
    if (expand) orow = load_row(a.out_rows + vv);
    free_job(a, (int)slot);
    st.c[kStAffected] += fresh ? 1ull : 0ull;  // lane 0 only
    st.c[kStExpansions] += expand ? 1ull : 0ull;
  }
  const int done = finish_vertices(a, vv, expand, requeue, orow, lane, s_excl, s_off, pb, st);
  note_done(a, vv, lane);
  return done;
}

// Mark token: marks one chunk of a vertex's out-row.
template <class P>
__device__ void run_mark_token(const Args<P>& a, unsigned u, unsigned chunk, int lane, PushBuf pb,
                               WarpStats& st) {
  const RowDesc r = load_row(a.out_rows + u);
  const long long beg = (long long)chunk * a.mark_split;
  const long long end = min((long long)r.deg, beg + a.mark_split);
  for (long long e0 = beg; e0 < end; e0 += 32 * kUnroll) {
    int t[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const long long e = e0 + k * 32 + lane;
      t[k] = e < end ? __ldg(a.out_edges + r.off + e) : -1;
    }
    unsigned wv[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) wv[k] = t[k] >= 0 ? ld_volatile(a.state + (t[k] >> 4)) : 0u;
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      if (e0 + k * 32 >= end) break;  // warp-uniform
      buf_push(a, pb, t[k], mark_one(a, t[k], t[k] >= 0 && !(P::closed_form && t[k] == (int)u), wv[k]),
               true, lane, st);
    }
  }
  if (lane == 0) st.c[kStMarked] += (unsigned long long)max(0ll, end - beg);
  buf_flush(a, pb, lane, st);
}

// ---------------------------------------------------------------------------
// Helping: the claimed vertices of a warp that stopped go back to the queue
// ---------------------------------------------------------------------------

// Every warp of a worklist launch keeps a hold record of kHoldWords 64-bit
// words: [0] its claim word, launch generation << 32 | claim epoch << 1 |
// holding; [1] a claim word a helper saw; [2] that helper's warp << 32 | its
// scan count; [3] the time of that sighting; [4..19] the 32 vertex ids of the
// warp's current batch. A warp publishes its batch right after claiming it
// and clears the holding bit once the batch is finished. An idle warp scans
// the records every kHelpScanEvery idle polls. A claim that the same helper
// saw unchanged in two of its scans, at least kHelpAfterNs apart, belongs to
// a warp that stopped (a batch takes well under a millisecond): the helper
// takes the record with a compare-and-swap and puts its vertices back in the
// queue with their open-work units. Both conditions are needed: the scan
// count does not advance while the device is paused, and the clock does.
constexpr int kHoldWords = 20;
constexpr unsigned kHelpScanEvery = 4096;
constexpr unsigned long long kHelpAfterNs = 10000000ull;

// This warp's hold record.
template <class P>
__device__ __forceinline__ unsigned long long* hold_of(const Args<P>& a, int w) {
  return a.hold + ((size_t)blockIdx.x * kWPB + (size_t)w) * kHoldWords;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

template <class P>
__device__ __forceinline__ void help_stopped_warps(const Args<P>& a, unsigned long long gen, int me,
                                                unsigned scan, int lane, PushBuf pb, WarpStats& st) {
  const int warps = (int)gridDim.x * kWPB;
  for (int base = 0; base < warps; base += 32) {
    const int r = base + lane;
    bool take = false;
    if (r < warps && r != me) {
      unsigned long long* rec = a.hold + (size_t)r * kHoldWords;
      const unsigned long long word = ld_volatile_u64(rec);
      if ((word >> 32) == gen && (word & 1ull)) {
        const unsigned long long seen = ld_volatile_u64(rec + 1);
        const unsigned long long who = ld_volatile_u64(rec + 2);
        const unsigned long long now = gtime();
        const unsigned long long since = now - ld_volatile_u64(rec + 3);
        if (seen != word || ((int)(who >> 32) != me && since > 3 * kHelpAfterNs)) {
          // first sighting of this claim (or its helper stopped too): note it
          *(volatile unsigned long long*)(rec + 1) = word;
          *(volatile unsigned long long*)(rec + 2) = ((unsigned long long)me << 32) | scan;
          *(volatile unsigned long long*)(rec + 3) = now;
        } else if ((int)(who >> 32) == me && scan - (unsigned)who >= 2u && since >= kHelpAfterNs) {
          take = atomicCAS(rec, word, word & ~1ull) == word;
        }
      }
    }
    unsigned todo = __ballot_sync(kFull, take);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int* ids = reinterpret_cast<const int*>(a.hold + (size_t)(base + src) * kHoldWords + 4);
      int v = ld_volatile(ids + lane);
      if (v >= a.n) v = -1;  // only ids of this graph were ever published
      if (v >= 0) {  // running (perhaps flagged) -> queued; its unit goes with it
        const unsigned sh = (unsigned)(v & 15) * 2u;
        atomicOr(a.state + (v >> 4), 1u << sh);
        atomicAnd(a.state + (v >> 4), ~(2u << sh));
      }
      __threadfence();
      buf_push(a, pb, v, v >= 0, false, lane, st);
      buf_flush(a, pb, lane, st);
    }
  }
}

template <class P>
__global__ void __launch_bounds__(kNT, 5) k_worklist(Args<P> a) {
  __shared__ int s_excl[kWPB][32];
  __shared__ long long s_off[kWPB][32];
  __shared__ typename P::acc s_acc[kWPB][32];
  __shared__ int s_push[kWPB][kPushCap];
  __shared__ int s_pcnt[kWPB][3];
  __shared__ unsigned long long s_stat[kWPB][kStCount];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  DfCtl* ctl = a.ctl;
  WarpStats st;
  stats_init(st, s_stat[w], lane);
  if (lane == 0) {
    s_pcnt[w][0] = 0;
    s_pcnt[w][1] = 0;
    s_pcnt[w][2] = 0;
  }
  __syncwarp();
  unsigned long long* const sc = s_stat[w];  // lane 0: counters; kStProcessed = recomputations
                                             // not yet added to the work-cap count
  const PushBuf pb{s_push[w], &s_pcnt[w][0], &s_pcnt[w][1], &s_pcnt[w][2]};
  // helping: the launch generation that tells this launch's hold records
  // from earlier ones, and this warp's claim epoch, idle polls and scans
  // (shared memory: they hold no registers)
  __shared__ unsigned long long s_gen;
  __shared__ unsigned s_help[kWPB][3];
  if (a.helping) {
    if (threadIdx.x == 0) s_gen = (ctl->t_start >> 10) & 0xffffffffull;
    if (lane == 0) {
      s_help[w][0] = s_help[w][1] = s_help[w][2] = 0u;
    }
    __syncthreads();
    if (lane == 0) *(volatile unsigned long long*)hold_of(a, w) = s_gen << 32;
  }
  auto mark = [&](int t, bool valid) {
    const unsigned word = valid ? ld_volatile(a.state + (t >> 4)) : 0u;
    const bool need = mark_one(a, t, valid, word);
    buf_push(a, pb, t, need, true, lane, st);
  };

  // Stage 1: initial marking. Each item holds one unit of `pending` until its
  // insertions are in the ring, so the iteration cannot end while marking is open.
  const unsigned long long n_items = ctl->n_items;
  while (true) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ctl->mark_next.v, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= n_items) break;
    do_mark_item(a, (long long)item, lane, st, mark);
    buf_flush(a, pb, lane, st);
    if (lane == 0) *pb.owed += 1;  // the item's own unit, settled later
    __syncwarp();
  }

  // Stage 2: chunk tokens first (they finish heavy vertices), then batches of
  // queued vertices, until nothing is queued, running or tokenised.
  unsigned backoff = 32;
  if (lane == 0) sc[kStClock] = (unsigned long long)clock64();
  auto phase_mark = [&](int ph) {  // lane 0 charges the time since the last mark to `ph`
    if (lane == 0) {
      const unsigned long long t = (unsigned long long)clock64();
      sc[kStPhase0 + ph] += t - sc[kStClock];
      sc[kStClock] = t;
    }
  };
  unsigned polls = 0;
  while (!a.mark_only) {
    // the stop conditions are also polled while work remains: a queue that
    // does not drain must still end at the work cap or the time budget
    if ((++polls & 15u) == 0u) {
      int stop = 0;
      if (lane == 0) {
        if (ld_volatile(&ctl->abort)) stop = 1;
        else if (timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          stop = 1;
        }
      }
      if (__shfl_sync(kFull, stop, 0)) break;
    }
    const unsigned long long tok = pop_token(a, lane);
    if (tok != kNoToken) {
      const unsigned kind = (unsigned)(tok >> 62);
      const unsigned x = (unsigned)((tok >> 31) & 0x7fffffffull);
      const unsigned y = (unsigned)(tok & 0x7fffffffull);
      phase_mark(1);
      int done = 0;
      if (kind == 0) done = run_gather_token(a, x, y, lane, s_excl[w], s_off[w], pb, st);
      else run_mark_token(a, x, y, lane, pb, st);
      if (lane == 0) {
        *pb.owed += 1 + done;  // the token's unit (and the finished vertex's)
        sc[kStTokens] += 1ull;
        sc[kStProcessed] += (unsigned long long)done;
      }
      __syncwarp();
      phase_mark(kind == 0 ? 2 : 3);
      continue;
    }
    // claim up to 32 items
    long long got = 0;
    unsigned long long h = 0;
    if (lane == 0) {
      if (ld_volatile(&ctl->avail.v) > 0) {
        const long long av = atomic_add_ll_old(&ctl->avail.v, -32);
        got = av >= 32 ? 32 : (av > 0 ? av : 0);
        if (got < 32) atomic_add_ll(&ctl->avail.v, 32 - got);
        if (got) h = atomicAdd(&ctl->head.v, (unsigned long long)got);
      }
    }
    got = __shfl_sync(kFull, got, 0);
    if (got == 0) {
      settle_owed(a, pb, lane);
      int stop = 0;
      if (lane == 0) {
        if (sc[kStProcessed]) {
          atomicAdd(&ctl->processed.v, sc[kStProcessed]);
          sc[kStProcessed] = 0;
        }
        if (ld_volatile(&ctl->abort) || ld_volatile(&ctl->pending.v) <= 0) stop = 1;
        else if (timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          stop = 1;
        }
      }
      if (__shfl_sync(kFull, stop, 0)) break;
      if (a.helping) {
        unsigned scan = 0;
        if (lane == 0 && ++s_help[w][1] % kHelpScanEvery == 0u) scan = ++s_help[w][2];
        scan = __shfl_sync(kFull, scan, 0);
        if (scan) help_stopped_warps(a, s_gen, (int)blockIdx.x * kWPB + w, scan, lane, pb, st);
      }
      __nanosleep(backoff);
      backoff = min(backoff * 2, 1024u);
      phase_mark(0);
      continue;
    }
    backoff = 32;
    if (lane == 0) sc[kStBatches] += 1;
    h = __shfl_sync(kFull, h, 0);
    int v = -1;
    bool ok = true;
    if (lane < got) {
      int* slot = a.queue + ((h + lane) & a.qmask);
      unsigned spins = 0;
      while ((v = ld_volatile(slot)) < 0) {  // producer between claim and write
        if ((++spins & 255u) == 0 && timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      if (ok) {
        *(volatile int*)slot = -1;
        const unsigned sh = (unsigned)(v & 15) * 2u;
        atomicXor(a.state + (v >> 4), 3u << sh);  // queued -> running
      } else {
        v = -1;
      }
    }
    if (!__all_sync(kFull, ok)) break;
    if (a.helping) {  // publish the batch (after settling this warp's earlier completions)
      settle_owed(a, pb, lane);
      unsigned long long* my = hold_of(a, w);
      reinterpret_cast<int*>(my + 4)[lane] = v;
      __syncwarp();
      if (lane == 0)
        *(volatile unsigned long long*)my = (s_gen << 32) | ((unsigned long long)(++s_help[w][0] & 0x7fffffffu) << 1) | 1ull;
    }
    if (a.fault_crash_warps &&
        fault_crash(a, __shfl_sync(kFull, lane == 0 ? sc[kStBatches] : 0ull, 0)))
      return;  // crash-stop holding claimed vertices (Sec. 5.4)
    __threadfence();  // state change before reading neighbours' contributions

    // the vertex's record: rank, x, in-row, out-degree, flags in one sector
    typename P::val r_old = 0, x_prev = 0;
    long long ioff = 0;
    int ideg = 0, od = 0;
    unsigned fl = 0;
    if (v >= 0) P::load_rec(a.rec + v, r_old, x_prev, ioff, ideg, od, fl);
    // Heavy in-rows become jobs of gather tokens that any warp can take; the
    // vertex stays running (and keeps its pending unit) until its last chunk.
    {
      int nch = 0, slot = -1;
      if (v >= 0) {
        const int din = ideg;
        if (din > a.gather_split) {
          slot = alloc_job(a);
          if (slot >= 0) {
            nch = (din + a.gather_split - 1) / a.gather_split;
            a.job_v[slot] = v;
            a.job_sum[slot] = 0ull;
            a.job_rem[slot] = nch;
            fence_acq_rel();
          }
        }
      }
      const unsigned jobs_b = __ballot_sync(kFull, nch > 0);
      if (jobs_b) {
        push_tokens(a, nch, 0u, (unsigned)max(slot, 0), lane, st, &ctl->pending.v);
        if (lane == 0) sc[kStJobs] += (unsigned long long)__popc(jobs_b);
        if (nch > 0) v = -1;
      }
    }
    phase_mark(1);

    const typename P::acc acc = gather_row(a, v >= 0 ? ideg : 0, ioff, lane, s_excl[w], s_off[w],
                                           s_acc[w], st);
    const double dangling = a.teleport ? ctl->dsum : 0.0;
    bool expand = false, requeue = false, fresh = false;
    RowDesc orow;
    orow.off = 0;
    orow.deg = 0;
    if (v >= 0) {
      vertex_epilogue_rec(a, v, P::total(acc), r_old, x_prev, fl, od, dangling, expand, requeue,
                          fresh, st);
      if (expand) orow = load_row(a.out_rows + v);  // the out-row's offset: expansions only
    }
    stats_count(st, kStAffected, fresh, lane);
    stats_count(st, kStExpansions, expand, lane);
    phase_mark(2);
    const int done = finish_vertices(a, v, expand, requeue, orow, lane, s_excl[w], s_off[w], pb, st);
    if (a.helping && lane == 0)  // the batch is finished: no longer holding
      *(volatile unsigned long long*)hold_of(a, w) =
          (s_gen << 32) | ((unsigned long long)(s_help[w][0] & 0x7fffffffu) << 1);
    note_done(a, v, lane);
    phase_mark(3);
    const unsigned proc_b = __ballot_sync(kFull, v >= 0);
    if (lane == 0) {
      *pb.owed += done;  // subtracted with the next flush or when idle
      const unsigned long long lp = sc[kStProcessed] + (unsigned long long)__popc(proc_b);
      sc[kStProcessed] = lp;
      if (lp >= 2048) {
        const unsigned long long pr = atomicAdd(&ctl->processed.v, lp);
        if ((long long)(pr + lp) > ctl->work_cap) stop_with(a, DFPR_ENOTCONV);
        sc[kStProcessed] = 0;
      }
    }
    __syncwarp();
    phase_mark(4);
    if (a.fault_delay_thr)
      fault_delay(a, __shfl_sync(kFull, lane == 0 ? sc[kStBatches] : 0ull, 0), v >= 0, lane);
  }
  settle_owed(a, pb, lane);
  if (lane == 0) {
    if (sc[kStProcessed]) atomicAdd(&ctl->processed.v, sc[kStProcessed]);
    if (sc[kStTokens]) atomicAdd(&ctl->tokens, sc[kStTokens]);
    if (sc[kStJobs]) atomicAdd(&ctl->jobs, sc[kStJobs]);
    if (sc[kStBatches]) atomicAdd(&ctl->batches, sc[kStBatches]);
    for (int i = 0; i < 5; ++i)
      if (sc[kStPhase0 + i]) atomicAdd(&ctl->phase[i], sc[kStPhase0 + i]);
  }
  flush_stats(a, st, lane);
}

// ---------------------------------------------------------------------------
// Round schedule (Alg. 2)
// ---------------------------------------------------------------------------

// Marks t affected (appending it to the affected list once) and not converged.
template <class P>
__device__ void mark_round(const Args<P>& a, int t, bool valid, int lane) {
  bool fresh = false;
  long long nc_add = 0;
  if (valid) {
    const uint32_t bit = 1u << (t & 31);
    // affected bits only grow during a call: a set bit needs no atomic
    if ((ld_volatile(a.va_bits + (t >> 5)) & bit) == 0u)
      fresh = (atomicOr(a.va_bits + (t >> 5), bit) & bit) == 0u;
    nc_add = (atomicOr(a.rc_bits + (t >> 5), bit) & bit) == 0u ? 1 : 0;
  }
  const unsigned b = __ballot_sync(kFull, fresh);
  const unsigned nb = __ballot_sync(kFull, nc_add != 0);
  long long base = 0;
  if (lane == 0) {
    if (nb) atomic_add_ll(&a.ctl->nc.v, __popc(nb));
    if (b) base = atomic_add_ll_old(&a.ctl->len.v, __popc(b));
  }
  base = __shfl_sync(kFull, base, 0);
  if (fresh) *(volatile int*)(a.alist + base + __popc(b & lanemask_lt())) = t;
}

// Alg. 2 epilogue for each lane's vertex v (or -1), from sum = the sum of its
// in-neighbours' contributions: writes R and C; when the change exceeds
// tau_f, marks the out-neighbours affected and not converged (with
// self-loops this flags v itself); when it is at most tau, clears v's R_C
// flag; then ends v's exclusion. Warp-uniform. Returns whether this lane
// cleared a flag.
template <class P>
__device__ bool round_finish(const Args<P>& a, int v, double sum, int lane, int* s_excl,
                             long long* s_off, WarpStats& st) {
  bool expand = false;
  double dr = 0.0, thr = 0.0;
  if (v >= 0) {
    const typename P::val r = (typename P::val)(base_of(a, v) + a.alpha * sum);
    const typename P::val r_old = P::load(a.R + v);
    dr = fabs((double)r - (double)r_old);
    const int od = a.out_rows[v].deg;
    a.R[v] = r;
    a.C[v] = contrib_of(r, od);
    const double thr_f = frontier_thr<P>(a.tol_f, r);
    thr = P::relative ? a.tol * fabs((double)r) : a.tol;
    expand = dr > thr_f;
    st.max_change = fmax(st.max_change, dr);
  }
  stats_count(st, kStExpansions, expand, lane);
  // expansion first (with self-loops it flags v itself), then v's own flag
  {
    int od = 0;
    long long oo = 0;
    if (expand) {
      const RowDesc r = a.out_rows[v];
      od = r.deg;
      oo = r.off;
    }
    int incl = od;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    s_excl[lane] = incl - od;
    s_off[lane] = oo;
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
      const int e = base + lane;
      const bool valid = e < total;
      int t = 0;
      if (valid) {
        const int o = owner_of(s_excl, e);
        t = a.out_edges[s_off[o] + (e - s_excl[o])];
      }
      mark_round(a, t, valid, lane);
    }
    if (lane == 0) st.c[kStMarked] += (unsigned long long)total;
  }
  bool conv = false;
  if (v >= 0 && dr <= thr) {
    const uint32_t bit = 1u << (v & 31);
    conv = (atomicAnd(a.rc_bits + (v >> 5), ~bit) & bit) != 0u;
  }
  if (v >= 0) {
    __threadfence();
    const unsigned sh = (unsigned)(v & 15) * 2u;
    atomicAnd(a.state + (v >> 4), ~(2u << sh));
  }
  return conv;
}

// Round schedule: a gather token (a chunk of a heavy vertex's in-row); the
// warp that sums the last chunk finishes the vertex with round_finish.
template <class P>
__device__ void round_gather_token(const Args<P>& a, unsigned slot, unsigned chunk, int lane,
                                   int* s_excl, long long* s_off, WarpStats& st) {
  int v = -1;
  if (sum_gather_token(a, slot, chunk, lane, st, &v)) {
    fence_acq_rel();
    double sum = 0.0;
    if (lane == 0) sum = P::job_total(ld_volatile(a.job_sum + slot));
    const bool conv = round_finish(a, lane == 0 ? v : -1, sum, lane, s_excl, s_off, st);
    if (lane == 0) {
      free_job(a, (int)slot);
      if (conv) atomic_add_ll(&a.ctl->nc.v, -1);
      atomicAdd(&a.ctl->processed.v, 1ull);
    }
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();  // the chunk's sum (and a finished vertex) before the count drops
    atomic_add_ll(&a.ctl->open_tokens.v, -1);
  }
  __syncwarp();
}

template <class P>
__global__ void __launch_bounds__(kNT) k_round(Args<P> a) {
  __shared__ int s_excl[kWPB][32];
  __shared__ long long s_off[kWPB][32];
  __shared__ typename P::acc s_acc[kWPB][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  DfCtl* ctl = a.ctl;
  __shared__ unsigned long long s_stat[kWPB][kStCount];
  WarpStats st;
  stats_init(st, s_stat[w], lane);
  auto mark = [&](int t, bool valid) { mark_round(a, t, valid, lane); };

  // Marking phase with helping (Alg. 2 marking loop): claim items; then, until
  // every item is done, redo items that are still open (idempotent).
  const unsigned long long n_items = ctl->n_items;
  while (true) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ctl->mark_next.v, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= n_items) break;
    do_mark_item(a, (long long)item, lane, st, mark);
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      if (atomicExch(a.item_done + item, 1u) == 0u) atomic_add_ll(&ctl->pending.v, -1);
    }
  }
  {
    unsigned long long scan = (unsigned long long)(blockIdx.x * kWPB + w);
    const unsigned long long stride = (unsigned long long)gridDim.x * kWPB;
    unsigned spins = 0;
    while (true) {
      int stop = 0;
      if (lane == 0) {
        if (ld_volatile(&ctl->pending.v) <= 0 || ld_volatile(&ctl->abort)) stop = 1;
        else if ((++spins & 63u) == 0 && timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          stop = 1;
        }
      }
      if (__shfl_sync(kFull, stop, 0)) break;
      const unsigned long long item = scan % n_items;
      scan += stride;
      if (ld_volatile(a.item_done + item) == 0u) {  // help an unfinished item
        do_mark_item(a, (long long)item, lane, st, mark);
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          if (atomicExch(a.item_done + item, 1u) == 0u) atomic_add_ll(&ctl->pending.v, -1);
        }
      }
    }
  }
  if (a.mark_only || ld_volatile(&ctl->abort)) {
    flush_stats(a, st, lane);
    return;
  }

  // Passes (Alg. 2 iteration loop).
  int pass = 0;
  unsigned long long fk = 0;  // chunks this warp has taken (fault simulation)
  for (; pass < a.max_iter; ++pass) {
    while (true) {
      {  // chunks of heavy gathers first: they finish vertices other warps wait on
        const unsigned long long tok = pop_token(a, lane);
        if (tok != kNoToken) {
          round_gather_token(a, (unsigned)((tok >> 31) & 0x7fffffffull),
                             (unsigned)(tok & 0x7fffffffull), lane, s_excl[w], s_off[w], st);
          continue;
        }
      }
      unsigned long long c = 0;
      long long len = 0;
      if (lane == 0) {
        c = atomicAdd(a.pass_ctr + pass, 32ull);
        len = ld_volatile(&ctl->len.v);
      }
      c = __shfl_sync(kFull, c, 0);
      len = __shfl_sync(kFull, len, 0);
      if ((long long)c >= len) break;
      const long long j = (long long)c + lane;
      int v = -1;
      bool ok = true;
      if (j < len) {
        unsigned spins = 0;
        while ((v = ld_volatile(a.alist + j)) < 0) {  // appended but not yet written
          if ((++spins & 255u) == 0 && timed_out(a)) {
            stop_with(a, DFPR_ETIMEOUT);
            ok = false;
            break;
          }
          __nanosleep(32);
        }
        if (!ok) v = -1;
      }
      if (!__all_sync(kFull, ok)) break;
      if (fault_crash(a, fk)) return;  // crash-stop holding a claimed chunk (Sec. 5.4)
      // Exclusion: a vertex another warp is recomputing right now (a warp in
      // a neighbouring pass) is skipped, so a result computed from older
      // neighbour ranks never overwrites a fresher one.
      if (v >= 0) {
        const unsigned sh = (unsigned)(v & 15) * 2u;
        if (atomicOr(a.state + (v >> 4), 2u << sh) & (2u << sh)) v = -1;
      }
      __threadfence();
      RowDesc irow;
      irow.off = 0;
      irow.deg = 0;
      if (v >= 0) irow = load_row(a.in_rows + v);
      // Heavy in-rows become jobs of gather tokens that any warp can take
      // (taken before new chunks); the vertex stays excluded until the warp
      // that sums its last chunk finishes it.
      {
        int nch = 0, slot = -1;
        if (v >= 0 && irow.deg > a.gather_split) {
          slot = alloc_job(a);
          if (slot >= 0) {
            nch = (irow.deg + a.gather_split - 1) / a.gather_split;
            a.job_v[slot] = v;
            a.job_sum[slot] = 0ull;
            a.job_rem[slot] = nch;
            fence_acq_rel();
          }
        }
        if (__ballot_sync(kFull, nch > 0)) {
          push_tokens(a, nch, 0u, (unsigned)max(slot, 0), lane, st, &ctl->open_tokens.v);
          if (nch > 0) {
            v = -1;
            irow.deg = 0;
          }
        }
      }
      const typename P::acc acc = gather_row(a, irow.deg, irow.off, lane, s_excl[w], s_off[w],
                                             s_acc[w], st);
      const long long conv = round_finish(a, v, P::total(acc), lane, s_excl[w], s_off[w], st) ? 1 : 0;
      const unsigned cb = __ballot_sync(kFull, conv != 0);
      const unsigned pb_ = __ballot_sync(kFull, v >= 0);
      if (lane == 0) {
        if (cb) atomic_add_ll(&ctl->nc.v, -(long long)__popc(cb));
        atomicAdd(&ctl->processed.v, (unsigned long long)__popc(pb_));
      }
      fault_delay(a, fk, v >= 0, lane);
      ++fk;
    }
    // End of this warp's pass: stop when nothing is flagged and no heavy
    // gather is open; go on to the next pass while something is flagged;
    // otherwise help with the open gathers (their vertices may flag more).
    int next = 0;
    while (true) {
      int act = 0;  // 0: help with tokens, 1: stop, 2: next pass
      if (lane == 0) {
        if (ld_volatile(&ctl->abort)) {
          act = 1;
        } else if (ld_volatile(&ctl->nc.v) > 0) {
          act = 2;
          if (timed_out(a)) {
            stop_with(a, DFPR_ETIMEOUT);
            act = 1;
          }
        } else if (ld_volatile(&ctl->open_tokens.v) <= 0) {
          act = 1;
        } else if (timed_out(a)) {
          stop_with(a, DFPR_ETIMEOUT);
          act = 1;
        }
      }
      act = __shfl_sync(kFull, act, 0);
      if (act != 0) {
        next = act == 2;
        break;
      }
      const unsigned long long tok = pop_token(a, lane);
      if (tok != kNoToken)
        round_gather_token(a, (unsigned)((tok >> 31) & 0x7fffffffull), (unsigned)(tok & 0x7fffffffull),
                           lane, s_excl[w], s_off[w], st);
      else
        __nanosleep(256);
    }
    if (!next) {
      ++pass;
      break;
    }
  }
  if (lane == 0) atomicMax(&ctl->passes, (unsigned long long)pass);
  flush_stats(a, st, lane);
}

// ---------------------------------------------------------------------------
// Jacobi schedule: one iteration over a vertex list (or all vertices)
// ---------------------------------------------------------------------------

// Jacobi schedule: whether v marks its out-neighbours now. The affected set
// only grows during a call and out-rows do not change, so once v has marked
// them all, marking them again changes nothing: v marks on its first
// expansion only (rc_bits, unused by this schedule, record it; they are
// cleared with the affected list at the end of the call).
template <class P>
__device__ __forceinline__ bool first_expansion(const Args<P>& a, int v) {
  const uint32_t bit = 1u << (v & 31);
  if (ld_volatile(a.rc_bits + (v >> 5)) & bit) return false;
  return (atomicOr(a.rc_bits + (v >> 5), bit) & bit) == 0u;
}

// Marks the out-neighbours of an expanding vertex (lane-local v, expand) as
// affected from the next iteration on: a bit in va_bits, and the affected
// list grows past the current count (warp-uniform call).
template <class P>
__device__ void jacobi_mark(const Args<P>& a, bool expand, int v, int lane, int* s_excl,
                            long long* s_off, WarpStats& st) {
  int od = 0;
  long long oo = 0;
  if (expand) {
    const RowDesc r = a.out_rows[v];
    od = r.deg;
    oo = r.off;
  }
  int incl = od;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  __syncwarp();
  s_excl[lane] = incl - od;
  s_off[lane] = oo;
  __syncwarp();
  for (int base = 0; base < total; base += 32) {
    const int e = base + lane;
    const bool valid = e < total;
    int t = 0;
    if (valid) {
      int lo = 0, hi = 32;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_excl[mid] <= e) lo = mid; else hi = mid;
      }
      t = a.out_edges[s_off[lo] + (e - s_excl[lo])];
    }
    // affected from the next iteration on: the list grows past `count`
    bool fresh = false;
    if (valid) {
      const uint32_t bit = 1u << (t & 31);
      // affected bits only grow during a call: a set bit needs no atomic
      if ((ld_volatile(a.va_bits + (t >> 5)) & bit) == 0u)
        fresh = (atomicOr(a.va_bits + (t >> 5), bit) & bit) == 0u;
    }
    const unsigned bb = __ballot_sync(kFull, fresh);
    long long base2 = 0;
    if (lane == 0 && bb) base2 = atomic_add_ll_old(&a.ctl->len.v, __popc(bb));
    base2 = __shfl_sync(kFull, base2, 0);
    if (fresh) a.alist[base2 + __popc(bb & lanemask_lt())] = t;
  }
  if (lane == 0) st.c[kStMarked] += (unsigned long long)total;
}

template <class P>
__global__ void __launch_bounds__(kNT) k_jacobi(Args<P> a, const typename P::val* __restrict__ Rin,
                                                const typename P::contrib* __restrict__ Cin,
                                                typename P::val* __restrict__ Rout,
                                                typename P::contrib* __restrict__ Cout,
                                                const int32_t* __restrict__ list, long long count,
                                                int frontier) {
  __shared__ int s_excl[kWPB][32];
  __shared__ long long s_off[kWPB][32];
  __shared__ typename P::acc s_acc[kWPB][32];
  __shared__ unsigned long long s_stat[kWPB][kStCount];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpStats st;
  stats_init(st, s_stat[w], lane);
  Args<P> b = a;
  b.C = const_cast<typename P::contrib*>(Cin);
  const long long nbatch = (count + 31) / 32;
  const double dangling = a.teleport ? a.ctl->dsum : 0.0;
  for (long long bi = (long long)blockIdx.x * kWPB + w; bi < nbatch; bi += (long long)gridDim.x * kWPB) {
    const long long j = bi * 32 + lane;
    int v = j < count ? (list ? list[j] : (int)j) : -1;
    RowDesc row;
    row.off = 0;
    row.deg = 0;
    if (v >= 0) row = load_row(a.in_rows + v);
    if (a.jh_v && row.deg > a.gather_split) {
      // a long in-row: summed in chunks by every warp of k_jacobi_heavy
      const long long slot = atomic_add_ll_old(&a.ctl->nheavy, 1);
      if (slot < a.jh_cap) {
        a.jh_v[slot] = v;
        a.jh_rem[slot] = (row.deg + a.gather_split - 1) / a.gather_split;
        a.jh_sum[slot] = 0ull;
        v = -1;
        row.deg = 0;
      }
    }
    const typename P::acc acc = gather_row(b, row.deg, row.off, lane, s_excl[w], s_off[w], s_acc[w], st);
    bool expand = false;
    if (v >= 0) {
      const typename P::val r = finish_rank(b, acc, dangling, v);
      const double dr = fabs((double)r - (double)Rin[v]);
      const int od = a.out_rows[v].deg;
      Rout[v] = r;
      Cout[v] = contrib_of(r, od);
      const double thr_f = frontier_thr<P>(a.tol_f, r);
      expand = frontier && dr > thr_f && first_expansion(a, v);
      st.max_change = fmax(st.max_change, dr);
    }
    stats_count(st, kStExpansions, expand, lane);
    if (frontier) jacobi_mark(a, expand, v, lane, s_excl[w], s_off[w], st);
    if (lane == 0) atomicAdd(&a.ctl->processed.v, (unsigned long long)min(32ll, count - bi * 32));
    fault_delay(a, (unsigned long long)bi, v >= 0, lane);
  }
  flush_stats(a, st, lane);
}

// Chunk offsets of the long in-rows registered by k_jacobi (one block):
// jh_off[h] = chunks of slots before h; the total goes to ctl->heavy_chunks.
__global__ void __launch_bounds__(1024) k_jacobi_heavy_scan(DfCtl* ctl, const int32_t* __restrict__ rem,
                                                            long long* __restrict__ off, long long cap) {
  __shared__ long long s_w[32];
  __shared__ long long s_carry;
  const long long nh = min(ctl->nheavy, cap);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) s_carry = 0;
  __syncthreads();
  for (long long base = 0; base < nh; base += 1024) {
    const long long i = base + t;
    const long long x = i < nh ? (long long)rem[i] : 0ll;
    long long incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      long long v = s_w[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += y;
      }
      s_w[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const long long before = (wid ? s_w[wid - 1] : 0ll) + s_carry;
    if (i < nh) off[i] = before + incl - x;
    __syncthreads();
    if (t == 0) s_carry += s_w[31];
    __syncthreads();
  }
  if (t == 0) ctl->heavy_chunks = s_carry;
}

// The long in-rows of a Jacobi iteration: every warp takes gather_split-edge
// chunks of them (grid-stride over all chunks), adds each chunk's sum into
// the row's slot, and the warp that adds the last chunk finishes the vertex
// (Eq. 1, change, frontier marking), as k_jacobi does for the rest.
template <class P>
__global__ void __launch_bounds__(kNT) k_jacobi_heavy(Args<P> a, const typename P::val* __restrict__ Rin,
                                                      const typename P::contrib* __restrict__ Cin,
                                                      typename P::val* __restrict__ Rout,
                                                      typename P::contrib* __restrict__ Cout,
                                                      int frontier) {
  __shared__ int s_excl[kWPB][32];
  __shared__ long long s_off[kWPB][32];
  __shared__ unsigned long long s_stat[kWPB][kStCount];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpStats st;
  stats_init(st, s_stat[w], lane);
  const long long nh = min(a.ctl->nheavy, a.jh_cap);
  const long long total = a.ctl->heavy_chunks;
  const double dangling = a.teleport ? a.ctl->dsum : 0.0;
  for (long long item = (long long)blockIdx.x * kWPB + w; item < total;
       item += (long long)gridDim.x * kWPB) {
    long long lo = 0, hi = nh;  // last slot h with jh_off[h] <= item
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (a.jh_off[mid] <= item) lo = mid; else hi = mid;
    }
    const int v = a.jh_v[lo];
    const RowDesc row = load_row(a.in_rows + v);
    const long long beg = (item - a.jh_off[lo]) * a.gather_split;
    const long long end = min((long long)row.deg, beg + a.gather_split);
    typename P::acc acc = P::zero();
    for (long long e0 = beg; e0 < end; e0 += 32 * kUnroll) {
      typename P::contrib xv[kUnroll];
      int uid[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const long long e = e0 + k * 32 + lane;
        uid[k] = e < end ? __ldg(a.in_edges + row.off + e) : -1;
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) xv[k] = uid[k] >= 0 ? P::load_c(Cin + uid[k]) : (typename P::contrib)0;
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) acc = P::add(acc, P::from(xv[k]));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = P::add(acc, P::shfl_xor(acc, d));
    int last = 0;
    if (lane == 0) {
      P::job_add(a.jh_sum + lo, acc);
      fence_acq_rel();
      last = atomicSub(a.jh_rem + lo, 1) == 1;
      st.c[kStEdges] += (unsigned long long)max(0ll, end - beg);
    }
    if (!__shfl_sync(kFull, last, 0)) continue;
    fence_acq_rel();
    bool expand = false;
    const int vv = lane == 0 ? v : -1;
    if (vv >= 0) {
      double sum = P::job_total(ld_volatile_u64(a.jh_sum + lo));
      if (a.teleport) sum += dangling / (double)a.n;
      const typename P::val r = (typename P::val)(base_of(a, vv) + a.alpha * sum);
      const double dr = fabs((double)r - (double)Rin[vv]);
      const int od = a.out_rows[vv].deg;
      Rout[vv] = r;
      Cout[vv] = contrib_of(r, od);
      expand = frontier && dr > frontier_thr<P>(a.tol_f, r) && first_expansion(a, vv);
      st.max_change = fmax(st.max_change, dr);
    }
    stats_count(st, kStExpansions, expand, lane);
    if (frontier) jacobi_mark(a, expand, vv, lane, s_excl[w], s_off[w], st);
  }
  flush_stats(a, st, lane);
}

// The affected list's new entries as sort keys, and back (Jacobi schedule:
// an iteration reads and writes separate vectors, so the order in which it
// visits the affected vertices is free; ascending ids keep rows and ranks of
// neighbouring list entries in the same sectors).
__global__ void k_list_widen(const int32_t* __restrict__ list, long long n,
                             unsigned long long* __restrict__ keys) {
  GRID_STRIDE(i, n) keys[i] = (unsigned long long)(unsigned)list[i];
}
__global__ void k_list_narrow(const unsigned long long* __restrict__ keys, long long n,
                              int32_t* __restrict__ list) {
  GRID_STRIDE(i, n) list[i] = (int32_t)keys[i];
}

// Initial marking for the Jacobi schedule: affected list + bitmap.
template <class P>
__global__ void __launch_bounds__(kNT) k_mark_list(Args<P> a) {
  __shared__ unsigned long long s_stat[kWPB][kStCount];
  const int lane = threadIdx.x & 31;
  WarpStats st;
  stats_init(st, s_stat[threadIdx.x >> 5], lane);
  auto mark = [&](int t, bool valid) {
    bool fresh = false;
    if (valid) {
      const uint32_t bit = 1u << (t & 31);
      // affected bits only grow during a call: a set bit needs no atomic
      if ((ld_volatile(a.va_bits + (t >> 5)) & bit) == 0u)
        fresh = (atomicOr(a.va_bits + (t >> 5), bit) & bit) == 0u;
    }
    const unsigned b = __ballot_sync(kFull, fresh);
    long long base = 0;
    if (lane == 0 && b) base = atomic_add_ll_old(&a.ctl->len.v, __popc(b));
    base = __shfl_sync(kFull, base, 0);
    if (fresh) a.alist[base + __popc(b & lanemask_lt())] = t;
  };
  const unsigned long long n_items = a.ctl->n_items;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long item = warp; item < (long long)n_items; item += nw) do_mark_item(a, item, lane, st, mark);
  flush_stats(a, st, lane);
}

// ---------------------------------------------------------------------------
// Small helper kernels
// ---------------------------------------------------------------------------

__global__ void k_mark_chunks(const int32_t* __restrict__ src, long long ns,
                              const RowDesc* __restrict__ out_rows, long long* cnt) {
  GRID_STRIDE(i, ns) {
    const long long d = out_rows[src[i]].deg;
    cnt[i] = d > 0 ? (d + kMarkChunk - 1) / kMarkChunk : 1;
  }
}

// k_mark_chunks over a capacity: entries at or past the device count *ns are 0
// (a replayed launch reads the current count).
__global__ void k_mark_chunks_cap(const int32_t* __restrict__ src, long long cap,
                                  const long long* __restrict__ ns,
                                  const RowDesc* __restrict__ out_rows, long long* cnt) {
  const long long n = *ns;
  GRID_STRIDE(i, cap) {
    long long c = 0;
    if (i < n) {
      const long long d = out_rows[src[i]].deg;
      c = d > 0 ? (d + kMarkChunk - 1) / kMarkChunk : 1;
    }
    cnt[i] = c;
  }
}

__global__ void k_init_ctl(DfCtl* c, const long long* n_src_items_dev, long long n_mark_dst,
                           long long work_cap, long long seeded, int count_items_pending,
                           int jobs, const long long* n_mark_dst_dev = nullptr) {
  const unsigned long long nsi = n_src_items_dev ? (unsigned long long)*n_src_items_dev : 0ull;
  if (n_mark_dst_dev) n_mark_dst = *n_mark_dst_dev;
  const unsigned long long items = nsi + (unsigned long long)((n_mark_dst + 31) / 32);
  DfCtl z;
  memset(&z, 0, sizeof z);
  z.n_src_items = nsi;
  z.n_items = items;
  z.n_mark_dst = n_mark_dst;
  z.pending.v = (count_items_pending ? (long long)items : 0) + seeded;
  z.tail.v = (unsigned long long)seeded;
  z.avail.v = seeded;
  z.work_cap = work_cap;
  z.len.v = 0;
  z.ftail.v = (unsigned long long)jobs;
  z.favail.v = jobs;
  z.t_start = gtime();
  *c = z;
}

// Fills the free ring of heavy-gather job slots with every slot id.
__global__ void k_init_jobs(int32_t* ring, int jobs) {
  GRID_STRIDE(i, jobs) ring[i] = (int32_t)i;
}

__global__ void k_seed_all(int32_t n, uint32_t* state, int32_t* queue) {
  GRID_STRIDE(i, n) {
    queue[i] = (int32_t)i;
    if ((i & 15) == 0) {
      const long long rem = n - i;
      state[i >> 4] = rem >= 16 ? 0x55555555u : (uint32_t)((1ull << (2 * rem)) - 1) & 0x55555555u;
    }
  }
}

// Per-vertex records of a worklist call from the ranks and row descriptors.
template <class P>
__global__ void k_build_rec(int32_t n, const RowDesc* __restrict__ in_rows,
                            const RowDesc* __restrict__ out_rows,
                            const typename P::val* __restrict__ R, VRec* rec) {
  GRID_STRIDE(v, n) {
    const RowDesc ir = load_row(in_rows + v);
    P::init_rec(rec + v, R[v], ir.off, ir.deg, out_rows[v].deg);
  }
}

// Ranks back from the records after a worklist call.
template <class P>
__global__ void k_rec_back(int32_t n, const VRec* __restrict__ rec, typename P::val* R) {
  GRID_STRIDE(v, n) R[v] = P::rec_rank(rec + v);
}

template <class T>
__global__ void k_fill(T* p, long long n, T v) {
  GRID_STRIDE(i, n) p[i] = v;
}

template <class T, class CT>
__global__ void k_init_ranks(int32_t n, const RowDesc* __restrict__ out_rows,
                             const int32_t* __restrict__ part_off, int nparts, T* R, CT* C) {
  GRID_STRIDE(u, n) {
    double nn = (double)n;
    if (nparts > 1) {
      const int p = part_of(part_off, nparts, (int)u);
      nn = (double)(part_off[p + 1] - part_off[p]);
    }
    const T r0 = (T)(1.0 / nn);
    R[u] = r0;
    C[u] = contrib_of(r0, out_rows[u].deg);
  }
}

// Flags in caller order: out[u] for internal vertex perm[u] (perm may be null).
__global__ void k_export_state(int32_t n, const uint32_t* __restrict__ state,
                               const int32_t* __restrict__ perm, uint8_t* out) {
  GRID_STRIDE(u, n) {
    const int v = perm ? perm[u] : (int)u;
    out[u] = ((state[v >> 4] >> ((v & 15) * 2)) & 3u) ? 1 : 0;
  }
}


// Clears the affected / not-converged bits of the listed vertices and the list.
__global__ void k_clear_list(int32_t* alist, long long len, uint32_t* va, uint32_t* rc) {
  GRID_STRIDE(i, len) {
    const int v = alist[i];
    if (v >= 0) {
      const uint32_t bit = 1u << (v & 31);
      if (va) atomicAnd(va + (v >> 5), ~bit);
      if (rc) atomicAnd(rc + (v >> 5), ~bit);
    }
    alist[i] = -1;
  }
}

template <class T>
__global__ void k_sum_ranks(int32_t n, const T* __restrict__ R, double* out) {
  __shared__ double sh[kWPB];
  double s = 0.0;
  GRID_STRIDE(i, n) s += (double)R[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kWPB; ++i) t += sh[i];
    atomicAdd(out, t);
  }
}

template <class T>
__global__ void k_dangling(int32_t n, const RowDesc* __restrict__ out_rows, const T* __restrict__ R,
                           double* out) {
  __shared__ double sh[kWPB];
  double s = 0.0;
  GRID_STRIDE(i, n) if (out_rows[i].deg == 0) s += (double)R[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kWPB; ++i) t += sh[i];
    atomicAdd(out, t);
  }
}

template <class T, class CT>
__global__ void k_scale(int32_t n, const RowDesc* __restrict__ out_rows, T* R, CT* C, const double* sum) {
  const double inv = 1.0 / *sum;
  GRID_STRIDE(u, n) {
    const T r = (T)((double)R[u] * inv);
    R[u] = r;
    C[u] = contrib_of(r, out_rows[u].deg);
  }
}

// ND / static round schedule: the affected list is every vertex, visited with
// a stride coprime to n so that the densest vertices (low internal ids) are
// spread over the pass instead of filling its first chunks.
__global__ void k_seed_round(int32_t n, long long stride, int32_t* alist, DfCtl* c) {
  GRID_STRIDE(i, n) alist[i] = (int32_t)(((long long)i * stride) % n);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->len.v = n;
    c->nc.v = n;
  }
}

// Residual of Eq. 1 at every vertex, in FP64 from the stored ranks (not the
// stored contributions): r'(v) = (1 - alpha) / n_v + alpha * (sum over in-edges
// (u, v) of R[u] / |out(u)| + dead / n), with n_v the vertex count of v's graph
// and dead the dead-end mass (0 with self-loops). A warp per vertex; the
// largest |r'(v) - R[v]| and |r'(v) - R[v]| / R[v] go to out[0] and out[1] as
// bit patterns (non-negative doubles order like their bits).
template <class T>
__global__ void k_residual(int32_t n, const RowDesc* __restrict__ in_rows,
                           const int32_t* __restrict__ in_edges,
                           const RowDesc* __restrict__ out_rows, const T* __restrict__ R,
                           const int32_t* __restrict__ part_off, int nparts, double alpha,
                           const double* dead, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const double tele = dead ? *dead / (double)n : 0.0;
  double worst = 0.0, worst_rel = 0.0;
  for (long long v = warp; v < n; v += nw) {
    const RowDesc row = load_row(in_rows + v);
    double s = 0.0;
    for (long long e = lane; e < row.deg; e += 32) {
      const int u = __ldg(in_edges + row.off + e);
      s += (double)R[u] / (double)out_rows[u].deg;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
    double nv = (double)n;
    if (nparts > 1) {
      const int p = part_of(part_off, nparts, (int)v);
      nv = (double)(__ldg(part_off + p + 1) - __ldg(part_off + p));
    }
    const double r = (1.0 - alpha) / nv + alpha * (s + tele);
    const double res = fabs(r - (double)R[v]);
    worst = fmax(worst, res);
    worst_rel = fmax(worst_rel, res / fabs((double)R[v]));
  }
  if (lane == 0) {
    if (worst > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(worst));
    if (worst_rel > 0.0) atomicMax(out + 1, (unsigned long long)__double_as_longlong(worst_rel));
  }
}

unsigned grid_small(long long n) { return blocks_for(n, kNT, sm_cap(16u)); }

// ---------------------------------------------------------------------------
// Host drivers
// ---------------------------------------------------------------------------

// SplitMix64 finaliser on the host (seeds the device-side fault draws).
unsigned long long host_mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <class P>
Args<P> make_args(dfpr_graph* g, const dfpr_params& p) {
  Args<P> a;
  memset(&a, 0, sizeof a);
  a.n = g->n;
  a.in_rows = g->in.rows.p;
  a.in_edges = g->in.edges.p;
  a.out_rows = g->out.rows.p;
  a.out_edges = g->out.edges.p;
  a.state = g->state.p;
  a.queue = g->queue.p;
  a.qmask = g->qcap - 1;
  a.ctl = g->ctl.p;
  a.tokens = g->tokens.p;
  a.tmask = g->tcap - 1;
  a.job_ring = g->job_ring.p;
  a.job_v = g->job_v.p;
  a.job_rem = g->job_rem.p;
  a.job_sum = g->job_sum.p;
  a.jmask = (unsigned)g->jcap - 1u;
  a.part_off = g->nparts > 1 ? g->part_off.p : nullptr;
  a.nparts = g->nparts;
  a.part_done = g->nparts > 1 ? g->part_done.p : nullptr;
  a.va_bits = g->va_bits.p;
  a.rc_bits = g->rc_bits.p;
  a.alist = g->affected_list.p;
  a.pass_ctr = g->pass_ctr.p;
  a.item_done = g->item_done.p;
  a.max_iter = p.max_iter;
  a.alpha = p.alpha;
  a.base = (1.0 - p.alpha) / (double)g->n;
  a.tol = p.tol;
  a.tol_f = p.frontier_tol > 0 ? p.frontier_tol : p.tol / 1000.0;
  a.teleport = g->cfg.dead_end == DFPR_TELEPORT;
  const double tmo = p.timeout_ms > 0 ? p.timeout_ms : 60000.0;
  a.timeout_ns = (unsigned long long)(tmo * 1e6);
  a.gather_split = p.gather_split > 0 ? p.gather_split : kGatherChunk;
  a.mark_split = p.mark_split > 0 ? p.mark_split : kMarkSplit;
  a.fault_seed = host_mix64(0x243f6a8885a308d3ull ^ (unsigned long long)p.fault_seed);
  a.fault_delay_thr = p.fault_delay_prob >= 1.0 ? ~0ull
                      : (unsigned long long)(p.fault_delay_prob * 18446744073709551616.0);
  a.fault_delay_ns = (unsigned long long)(p.fault_delay_us * 1000.0);
  a.fault_crash_warps = p.fault_crash_warps;
  a.hold = nullptr;
  a.helping = 0;
  a.jh_v = nullptr;
  a.jh_rem = nullptr;
  a.jh_sum = nullptr;
  a.jh_off = nullptr;
  a.jh_cap = 0;
  a.fault_perm_a = 1;
  a.fault_perm_b = 0;
  a.fault_warps = 1;
  return a;
}

// The crashing warps of a launch of `grid` CTAs: slot(w) = (w * A + B) mod W is
// a bijection of the W warps when gcd(A, W) = 1; warps with slot < the crash
// count crash.
template <class P>
void set_fault_warps(Args<P>& a, int grid) {
  const unsigned long long W = (unsigned long long)grid * kWPB;
  a.fault_warps = W;
  if (a.fault_crash_warps == 0) return;  // run_any checked fault_crash_warps < W
  unsigned long long A = (host_mix64(a.fault_seed ^ 1ull) % W) | 1ull;
  while (std::gcd(A, W) != 1ull) A = (A + 2) % W;
  a.fault_perm_a = A;
  a.fault_perm_b = host_mix64(a.fault_seed ^ 2ull) % W;
}

template <class P>
void set_vectors(dfpr_graph* g, Args<P>& a);
template <>
void set_vectors<P64>(dfpr_graph* g, Args<P64>& a) {
  a.R = g->R64.p;
  a.C = g->C64.p;
  a.rec = g->vrec.p;
}
template <>
void set_vectors<P32>(dfpr_graph* g, Args<P32>& a) {
  a.R = g->R32.p;
  a.C = g->C32.p;
  a.rec = g->vrec.p;
}

int persistent_grid(dfpr_graph* g, const dfpr_params& p, const void* kernel) {
  if (p.grid_ctas > 0) return p.grid_ctas;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kNT, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * g->sm_count;
}

// Grid of the worklist schedule: about sqrt(n) / 4 CTAs (at least 8), and at
// most 4 CTAs per SM (or the occupancy limit, if lower). Every warp holds 32
// vertices in flight; when the in-flight set is a large share of the
// frontier, vertices are recomputed from inputs that are about to change and
// are queued again. Measured on R-MAT graphs with 16 draws per vertex, batch
// 1e-4 |E|, FP64, ms per update (mean of 5-16 batches) at the grid given:
//  - scale 20: 128 / 192 / 256 / 320 / 384 CTAs: 24 / 17 / 16 / 15 / 16 ms;
//  - scale 22: 256 / 384 / 456 / 512 / 608 / 760: 31 / 33 / 30 / 24 / 35 / 38;
//  - scale 23: 380 / 456 / 532 / 608 / 760: 42 / 47 / 49 / 50 / 54;
//  - scale 24: 456 / 532 / 608 / 684 / 760: 84 / 70 / 55 / 69 / 75, the
//    same minimum on a second seed (54 against 76 ms) and at 1e-3 |E|
//    batches (90 against 99); at 1e-5 |E|, 65 against 63.
// The time follows the work: at 4 CTAs per SM the scale-24 updates did
// 5.3-8.4 n recomputations (10.1-10.6 n at 5 per SM), with fewer hub
// recomputations and expansions; the dependence on the grid is not monotone.
template <class P>
int worklist_grid(dfpr_graph* g, const dfpr_params& p) {
  const int full = persistent_grid(g, p, (const void*)k_worklist<P>);
  if (p.grid_ctas > 0) return full;
  const long long cap = std::min<long long>(full, 4ll * g->sm_count);
  const long long by_size = (long long)(0.25 * std::sqrt((double)g->n));
  return (int)std::max<long long>(std::min<long long>(8, cap), std::min<long long>(cap, by_size));
}

// Grid of the round schedule. One CTA per 2048 vertices at most: warps move
// to the next pass as soon as the current one's chunks are claimed, so the
// more vertices are in flight at once, the more each pass computes from
// stale neighbour ranks and the more passes convergence takes (R-MAT scale
// 14, 11.5K affected vertices: 2 / 4 / 8 / 16 CTAs took about 84 / 105 /
// 170 / 390 of the 500 passes, 48 / 30 / 22 / 22 ms).
template <class P>
int round_grid(dfpr_graph* g, const dfpr_params& p) {
  const int grid = persistent_grid(g, p, (const void*)k_round<P>);
  if (p.grid_ctas > 0) return grid;
  return (int)std::max<long long>(1, std::min<long long>(grid, (g->n + 2047) / 2048));
}

// Prepares marking items for the pending change set; returns the device
// pointer holding the number of source items.
template <class P>
long long* prepare_marking(dfpr_graph* g, Args<P>& a) {
  cudaStream_t s = g->stream;
  const long long ns = g->pend.n_src;
  long long* cnt = g->scratch.get<long long>(kSMarkCnt, (size_t)ns + 1, s);
  long long* off = g->scratch.get<long long>(kSMarkOff, (size_t)ns + 1, s);
  if (ns > 0) {
    k_mark_chunks<<<grid_small(ns), kNT, 0, s>>>(g->pend.src.p, ns, g->out.rows.p, cnt);
    DFPR_LAUNCHED();
  }
  scan_exclusive_i64(cnt, off, ns, off + ns, g->scratch, s);
  a.mark_src = g->pend.src.p;
  a.mark_choff = off;
  a.n_mark_src = ns;
  a.mark_dst = g->pend.dst.p;
  a.n_mark_dst = g->pend.n_dst;
  return off + ns;
}

struct CtlHost {
  DfCtl c;
};

CtlHost read_ctl(dfpr_graph* g) {
  CtlHost h;
  DFPR_CUDA(cudaMemcpyAsync(&h.c, g->ctl.p, sizeof(DfCtl), cudaMemcpyDeviceToHost, g->stream));
  DFPR_CUDA(cudaStreamSynchronize(g->stream));
  return h;
}

void fill_stats(const DfCtl& c, dfpr_stats* st) {
  st->processed = (int64_t)c.processed.v;
  st->edges_gathered = (int64_t)c.edges;
  st->expansions = (int64_t)c.expansions;
  st->edges_marked = (int64_t)c.edges_marked;
  st->pushes = (int64_t)c.pushes;
  st->affected = (int64_t)c.affected;
  double mc;
  memcpy(&mc, &c.max_change_bits, sizeof mc);
  st->residual_linf = mc;
  st->batches = (int64_t)c.batches;
  st->tokens = (int64_t)c.tokens;
  st->jobs = (int64_t)c.jobs;
  for (int i = 0; i < 5; ++i) st->phase_cycles[i] = (int64_t)c.phase[i];
}

// Resets the queue and states after an aborted worklist run.
void reset_worklist_state(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  DFPR_CUDA(cudaMemsetAsync(g->state.p, 0, sizeof(uint32_t) * g->state.count, s));
  k_fill<int32_t><<<grid_small((long long)g->qcap), kNT, 0, s>>>(g->queue.p, (long long)g->qcap, -1);
  DFPR_LAUNCHED();
  k_fill<unsigned long long><<<grid_small((long long)g->tcap), kNT, 0, s>>>(g->tokens.p, (long long)g->tcap, ~0ull);
  DFPR_LAUNCHED();
}

// Enqueues the device work of a DF update on the worklist schedule for a
// replayable CUDA graph: marking items over the capacity of the pending change
// set (the counts are read on the device, from a word the graph's first node
// copies from pinned host memory at every replay), the control block, the
// per-vertex records, the persistent kernel between two events, and the ranks
// copied back. Nothing here allocates or reads back.
template <class P>
void enqueue_captured_update(dfpr_graph* g, Args<P>& a, long long capn, long long* cnt,
                             long long* off, long long work_cap, int grid) {
  cudaStream_t s = g->stream;
  DFPR_CUDA(cudaMemcpyAsync(g->cap_dev.p, g->cap_host, 2 * sizeof(long long),
                            cudaMemcpyHostToDevice, s));
  k_mark_chunks_cap<<<grid_small(capn), kNT, 0, s>>>(g->pend.src.p, capn, g->cap_dev.p,
                                                     g->out.rows.p, cnt);
  DFPR_LAUNCHED();
  scan_exclusive_i64(cnt, off, capn, off + capn, g->cap_scratch, s);
  k_init_ctl<<<1, 1, 0, s>>>(g->ctl.p, off + capn, 0, work_cap, 0, 1, g->jcap, g->cap_dev.p + 1);
  DFPR_LAUNCHED();
  k_init_jobs<<<grid_small(g->jcap), kNT, 0, s>>>(g->job_ring.p, g->jcap);
  DFPR_LAUNCHED();
  if (g->nparts > 1)
    DFPR_CUDA(cudaMemsetAsync(g->part_done.p, 0, sizeof(unsigned long long) * g->nparts, s));
  k_build_rec<P><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->in.rows.p, g->out.rows.p, a.R, a.rec);
  DFPR_LAUNCHED();
  // external records: the replay records the events (a plain record inside a
  // capture only orders the captured work)
  DFPR_CUDA(cudaEventRecordWithFlags(g->cap_ev[0], s, cudaEventRecordExternal));
  k_worklist<P><<<grid, kNT, 0, s>>>(a);
  DFPR_LAUNCHED();
  DFPR_CUDA(cudaEventRecordWithFlags(g->cap_ev[1], s, cudaEventRecordExternal));
  k_rec_back<P><<<grid_small(g->n), kNT, 0, s>>>(g->n, a.rec, a.R);
  DFPR_LAUNCHED();
}

// The DF update's device work replayed from a CUDA graph (captured on first
// use, and again whenever a buffer, the grid or a parameter it was captured
// with changes). Returns the persistent kernel's time in *kernel_ms.
template <class P>
void run_captured_update(dfpr_graph* g, const dfpr_params& p, Args<P>& a, float* kernel_ms) {
  cudaStream_t s = g->stream;
  const long long capn = std::max<long long>(1, (long long)g->pend.src.count);
  long long* cnt = g->cap_scratch.get<long long>(0, (size_t)capn + 1, s);
  long long* off = g->cap_scratch.get<long long>(1, (size_t)capn + 1, s);
  // sizes the scan's level buffer outside the capture (no allocation may
  // happen inside it); the values are recomputed at every replay
  scan_exclusive_i64(cnt, off, capn, off + capn, g->cap_scratch, s);
  if (g->cap_dev.count < 2) g->cap_dev.reset(2, s);
  if (!g->cap_host) DFPR_CUDA(cudaMallocHost(&g->cap_host, 2 * sizeof(unsigned long long)));
  for (int i = 0; i < 2; ++i)
    if (!g->cap_ev[i]) DFPR_CUDA(cudaEventCreate(&g->cap_ev[i]));
  if (g->vrec.count < (size_t)g->n) g->vrec.reset(g->n, s);
  a.rec = g->vrec.p;
  a.mark_src = g->pend.src.p;
  a.mark_choff = off;
  a.n_mark_src = capn;  // padded items hold no chunks
  a.mark_dst = g->pend.dst.p;
  a.n_mark_dst = 0;     // read from the control block
  const int grid = worklist_grid<P>(g, p);
  set_fault_warps(a, grid);
  const long long work_cap = (long long)p.max_iter * (long long)g->n;
  // what the captured launches depend on
  std::vector<unsigned char> key(sizeof a);
  memcpy(key.data(), &a, sizeof a);
  const uintptr_t extra[] = {(uintptr_t)capn, (uintptr_t)cnt, (uintptr_t)off,
                             (uintptr_t)g->cap_scratch.buf[kSlotScanSums].p,
                             (uintptr_t)grid, (uintptr_t)g->part_done.p, (uintptr_t)g->nparts,
                             (uintptr_t)work_cap, (uintptr_t)g->pend.dst.p,
                             (uintptr_t)(g->cfg.precision), (uintptr_t)s};
  key.insert(key.end(), (const unsigned char*)extra, (const unsigned char*)extra + sizeof extra);
  if (!g->cap_exec || key != g->cap_key) {
    if (g->cap_exec) {
      DFPR_CUDA(cudaGraphExecDestroy(g->cap_exec));
      g->cap_exec = nullptr;
    }
    g->cap_host[0] = g->cap_host[1] = 0;
    const long long l0 = g_launches.load();
    DFPR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
      enqueue_captured_update<P>(g, a, capn, cnt, off, work_cap, grid);
    } catch (...) {
      cudaStreamEndCapture(s, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    DFPR_CUDA(cudaStreamEndCapture(s, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&g->cap_exec, graph, 0);
    cudaGraphDestroy(graph);
    DFPR_CUDA(ie);
    g->cap_launches = g_launches.load() - l0;
    g_launches.fetch_add(-g->cap_launches);  // counted at every replay instead
    g->cap_key.swap(key);
    ++g->cap_captures;
  }
  g->cap_host[0] = (unsigned long long)g->pend.n_src;
  g->cap_host[1] = (unsigned long long)g->pend.n_dst;
  DFPR_CUDA(cudaGraphLaunch(g->cap_exec, s));
  g_launches.fetch_add(g->cap_launches);
  ++g->cap_replays;
  DFPR_CUDA(cudaEventSynchronize(g->cap_ev[1]));
  DFPR_CUDA(cudaEventElapsedTime(kernel_ms, g->cap_ev[0], g->cap_ev[1]));
}

template <class P>
dfpr_status run_worklist(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st,
                         cudaEvent_t e0, cudaEvent_t e1, bool mark_only, float* kernel_ms = nullptr) {
  cudaStream_t s = g->stream;
  Args<P> a = make_args<P>(g, p);
  set_vectors<P>(g, a);
  a.mark_only = mark_only ? 1 : 0;
  if (p.helping && !mark_only) {  // hold records for every warp of the launch
    const size_t words = (size_t)worklist_grid<P>(g, p) * kWPB * kHoldWords;
    if (g->hold.count < words) {
      g->hold.reset(words, s);
      // a record is read only while its generation is this launch's; zeros
      // belong to no launch
      DFPR_CUDA(cudaMemsetAsync(g->hold.p, 0, words * sizeof(unsigned long long), s));
    }
    a.hold = g->hold.p;
    a.helping = 1;
  }
  if (g->capture && kind == kRunDF && !mark_only && !a.teleport && s != nullptr && kernel_ms) {
    run_captured_update<P>(g, p, a, kernel_ms);
  } else {
    long long* nsi = nullptr;
    long long seeded = 0;
    if (kind == kRunDF) {
      nsi = prepare_marking<P>(g, a);
    } else {
      seeded = g->n;
    }
    const long long work_cap = (long long)p.max_iter * (long long)g->n;
    k_init_ctl<<<1, 1, 0, s>>>(g->ctl.p, nsi, kind == kRunDF ? g->pend.n_dst : 0, work_cap, seeded, 1, g->jcap);
    DFPR_LAUNCHED();
    k_init_jobs<<<grid_small(g->jcap), kNT, 0, s>>>(g->job_ring.p, g->jcap);
    DFPR_LAUNCHED();
    if (seeded) {
      k_seed_all<<<grid_small(g->n), kNT, 0, s>>>(g->n, g->state.p, g->queue.p);
      DFPR_LAUNCHED();
    }
    if (a.teleport) {
      // the dead-end mass enters every vertex: computed once per call here
      DFPR_CUDA(cudaMemsetAsync(&g->ctl.p->dsum, 0, sizeof(double), s));
      k_dangling<typename P::val><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, a.R, &g->ctl.p->dsum);
      DFPR_LAUNCHED();
    }
    if (g->nparts > 1)
      DFPR_CUDA(cudaMemsetAsync(g->part_done.p, 0, sizeof(unsigned long long) * g->nparts, s));
    const int grid = worklist_grid<P>(g, p);
    if (!mark_only) {
      if (g->vrec.count < (size_t)g->n) g->vrec.reset(g->n, s);
      a.rec = g->vrec.p;
      k_build_rec<P><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->in.rows.p, g->out.rows.p, a.R, a.rec);
      DFPR_LAUNCHED();
    }
    DFPR_CUDA(cudaEventRecord(e0, s));  // the stats time the persistent kernel alone
    set_fault_warps(a, grid);
    k_worklist<P><<<grid, kNT, 0, s>>>(a);
    DFPR_LAUNCHED();
    DFPR_CUDA(cudaEventRecord(e1, s));
    if (!mark_only) {
      k_rec_back<P><<<grid_small(g->n), kNT, 0, s>>>(g->n, a.rec, a.R);
      DFPR_LAUNCHED();
    }
  }
  CtlHost h = read_ctl(g);
  if (st) fill_stats(h.c, st);
  if (g->nparts > 1 && !mark_only) {
    std::vector<unsigned long long> done((size_t)g->nparts);
    DFPR_CUDA(cudaMemcpyAsync(done.data(), g->part_done.p, sizeof(unsigned long long) * g->nparts,
                              cudaMemcpyDeviceToHost, s));
    DFPR_CUDA(cudaStreamSynchronize(s));
    g->part_ms.assign((size_t)g->nparts, 0.0);
    for (int i = 0; i < g->nparts; ++i)
      if (done[i] > h.c.t_start) g->part_ms[i] = (double)(done[i] - h.c.t_start) * 1e-6;
  }
  const bool clean = h.c.status == 0 && h.c.pending.v <= 0 && !mark_only;
  if (!clean && !mark_only) reset_worklist_state(g);
  return h.c.status ? (dfpr_status)h.c.status : DFPR_OK;
}

template <class P>
dfpr_status run_round(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st,
                      cudaEvent_t e0, cudaEvent_t e1) {
  cudaStream_t s = g->stream;
  Args<P> a = make_args<P>(g, p);
  set_vectors<P>(g, a);
  long long* nsi = nullptr;
  if (kind == kRunDF) nsi = prepare_marking<P>(g, a);
  DFPR_CUDA(cudaEventRecord(e0, s));
  k_init_ctl<<<1, 1, 0, s>>>(g->ctl.p, nsi, kind == kRunDF ? g->pend.n_dst : 0, 0, 0, 1, g->jcap);
  DFPR_LAUNCHED();
  k_init_jobs<<<grid_small(g->jcap), kNT, 0, s>>>(g->job_ring.p, g->jcap);
  DFPR_LAUNCHED();
  g->pass_ctr.ensure((size_t)p.max_iter + 1, s);
  a.pass_ctr = g->pass_ctr.p;
  DFPR_CUDA(cudaMemsetAsync(g->pass_ctr.p, 0, sizeof(unsigned long long) * (p.max_iter + 1), s));
  // marking-item completion flags (the helping rule)
  if (kind == kRunDF) {
    const long long nsrc_items = (long long)read_word(g, nsi, sizeof(long long));
    const long long items = nsrc_items + (g->pend.n_dst + 31) / 32;
    g->item_done.ensure((size_t)items + 1, s);
    a.item_done = g->item_done.p;
    DFPR_CUDA(cudaMemsetAsync(g->item_done.p, 0, sizeof(uint32_t) * (items + 1), s));
  } else {
    // ND / static: every vertex is affected and not converged from the start
    DFPR_CUDA(cudaMemsetAsync(g->va_bits.p, 0xff, sizeof(uint32_t) * g->va_bits.count, s));
    DFPR_CUDA(cudaMemsetAsync(g->rc_bits.p, 0xff, sizeof(uint32_t) * g->rc_bits.count, s));
    long long stride = ((long long)((double)g->n * 0.6180339887498949)) | 1;
    while (std::gcd(stride, (long long)g->n) != 1) stride += 2;
    k_seed_round<<<grid_small(g->n), kNT, 0, s>>>(g->n, stride % g->n == 0 ? 1 : stride,
                                                  g->affected_list.p, g->ctl.p);
    DFPR_LAUNCHED();
  }
  const int grid = round_grid<P>(g, p);
  set_fault_warps(a, grid);
  k_round<P><<<grid, kNT, 0, s>>>(a);
  DFPR_LAUNCHED();
  DFPR_CUDA(cudaEventRecord(e1, s));
  CtlHost h = read_ctl(g);
  if (st) {
    fill_stats(h.c, st);
    st->passes = (int32_t)h.c.passes;
    st->affected = h.c.len.v;
  }
  dfpr_status status = h.c.status ? (dfpr_status)h.c.status : DFPR_OK;
  if (status == DFPR_OK && h.c.nc.v > 0) status = DFPR_ENOTCONV;
  // a run that stopped early can leave exclusion bits and tokens behind
  if (h.c.status != 0 || h.c.open_tokens.v != 0) reset_worklist_state(g);
  // clear flags and list for the next call
  k_clear_list<<<grid_small(h.c.len.v), kNT, 0, s>>>(g->affected_list.p, h.c.len.v, g->va_bits.p, g->rc_bits.p);
  DFPR_LAUNCHED();
  if (kind != kRunDF) {
    DFPR_CUDA(cudaMemsetAsync(g->va_bits.p, 0, sizeof(uint32_t) * g->va_bits.count, s));
    DFPR_CUDA(cudaMemsetAsync(g->rc_bits.p, 0, sizeof(uint32_t) * g->rc_bits.count, s));
  }
  return status;
}

template <class T>
void swap_arrays(DevArray<T>& x, DevArray<T>& y) {
  std::swap(x.p, y.p);
  std::swap(x.count, y.count);
  std::swap(x.s, y.s);
  std::swap(x.rec, y.rec);
}

template <class P>
void swap_vectors(dfpr_graph* g);
template <>
void swap_vectors<P64>(dfpr_graph* g) {
  swap_arrays(g->R64, g->R64b);
  swap_arrays(g->C64, g->C64b);
}
template <>
void swap_vectors<P32>(dfpr_graph* g) {
  swap_arrays(g->R32, g->R32b);
  swap_arrays(g->C32, g->C32b);
}

template <class P>
void second_vectors(dfpr_graph* g, typename P::val** R2, typename P::contrib** C2);
template <>
void second_vectors<P64>(dfpr_graph* g, double** R2, long long** C2) {
  if (!g->R64b.p) {
    g->R64b.reset(g->n, g->stream);
    g->C64b.reset(g->n, g->stream);
  }
  *R2 = g->R64b.p;
  *C2 = g->C64b.p;
}
template <>
void second_vectors<P32>(dfpr_graph* g, float** R2, float** C2) {
  if (!g->R32b.p) {
    g->R32b.reset(g->n, g->stream);
    g->C32b.reset(g->n, g->stream);
  }
  *R2 = g->R32b.p;
  *C2 = g->C32b.p;
}

// Jacobi schedule: host loop of one kernel per iteration, L-inf stop test.
template <class P>
dfpr_status run_jacobi(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st,
                       cudaEvent_t e0, cudaEvent_t e1) {
  cudaStream_t s = g->stream;
  using V = typename P::val;
  using CV = typename P::contrib;
  V* R2 = nullptr;
  CV* C2 = nullptr;
  second_vectors<P>(g, &R2, &C2);
  Args<P> a = make_args<P>(g, p);
  set_vectors<P>(g, a);
  long long* nsi = nullptr;
  if (kind == kRunDF) nsi = prepare_marking<P>(g, a);
  DFPR_CUDA(cudaEventRecord(e0, s));
  k_init_ctl<<<1, 1, 0, s>>>(g->ctl.p, nsi, kind == kRunDF ? g->pend.n_dst : 0, 0, 0, 0, 0);
  DFPR_LAUNCHED();
  const bool df = kind == kRunDF;
  long long count = g->n;
  if (df) {
    // unaffected vertices keep R_prev in both vectors
    DFPR_CUDA(cudaMemcpyAsync(R2, a.R, sizeof(V) * g->n, cudaMemcpyDeviceToDevice, s));
    DFPR_CUDA(cudaMemcpyAsync(C2, a.C, sizeof(CV) * g->n, cudaMemcpyDeviceToDevice, s));
    k_mark_list<P><<<grid_small(32ll * g->n), kNT, 0, s>>>(a);
    DFPR_LAUNCHED();
    count = (long long)read_word(g, &g->ctl.p->len.v, sizeof(long long));
  }
  const int grid = persistent_grid(g, p, (const void*)k_jacobi<P>);
  // the jacobi schedule's own default chunk for long in-rows (R-MAT 24,
  // Static_BB: 200 ms at 4096-edge chunks, 131 ms at 2048, 450 at 16384)
  if (p.gather_split == 0) a.gather_split = kJacobiChunk;
  {  // slots for the long in-rows of an iteration: at most m / gather_split
    const long long cap = g->m / a.gather_split + 2;
    if ((long long)g->jh_v.count < cap) {
      g->jh_v.reset((size_t)cap, s);
      g->jh_rem.reset((size_t)cap, s);
      g->jh_sum.reset((size_t)cap, s);
      g->jh_off.reset((size_t)cap, s);
    }
    a.jh_v = g->jh_v.p;
    a.jh_rem = g->jh_rem.p;
    a.jh_sum = g->jh_sum.p;
    a.jh_off = g->jh_off.p;
    a.jh_cap = (long long)g->jh_v.count;
  }
  const unsigned long long fault_seed0 = a.fault_seed;
  // DF with teleport dead ends: every rank holds alpha * D / n, D the dead-end
  // mass. Ranks outside the affected set were computed with D_last; once the
  // current D differs from it by more than tol_f * n / alpha (relative to the
  // mean rank 1/n in FP32 mode), every vertex is recomputed from then on.
  // D_last starts at the mass the ranks had before the batch.
  const bool tdf = df && a.teleport;
  const double D_last = g->d_before_valid ? g->d_before : NAN;
  const double shift_tol = P::relative ? a.tol_f / (double)g->n : a.tol_f;
  bool all = false;
  int it = 0;
  double last = 0.0;
  bool converged = false;
  long long sorted_upto = 0;  // the list's prefix already in ascending id order
  int id_bits = 1;
  while (id_bits < 31 && (1ll << id_bits) < (long long)g->n) ++id_bits;
  for (; it < p.max_iter; ++it) {
    DFPR_CUDA(cudaMemsetAsync(&g->ctl.p->max_change_bits, 0, sizeof(unsigned long long), s));
    if (a.teleport) {
      DFPR_CUDA(cudaMemsetAsync(&g->ctl.p->dsum, 0, sizeof(double), s));
      k_dangling<V><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, a.R, &g->ctl.p->dsum);
      DFPR_LAUNCHED();
    }
    if (tdf && !all) {
      const unsigned long long bits = read_word(g, &g->ctl.p->dsum, sizeof(double));
      double D;
      memcpy(&D, &bits, sizeof D);
      if (!(p.alpha * std::fabs(D - D_last) / (double)g->n <= shift_tol)) all = true;  // NaN: unknown
    }
    const bool listed = df && !all;
    if (listed && count > sorted_upto) {  // entries appended since the last sort
      const long long k = count - sorted_upto;
      int32_t* seg = g->affected_list.p + sorted_upto;
      unsigned long long* keys = g->scratch.get<unsigned long long>(kSListKeys, (size_t)k, s);
      unsigned long long* tmp = g->scratch.get<unsigned long long>(kSListTmp, (size_t)k, s);
      k_list_widen<<<grid_small(k), kNT, 0, s>>>(seg, k, keys);
      DFPR_LAUNCHED();
      unsigned long long* sorted = radix_sort_u64(keys, tmp, k, id_bits, g->scratch, s);
      k_list_narrow<<<grid_small(k), kNT, 0, s>>>(sorted, k, seg);
      DFPR_LAUNCHED();
      sorted_upto = count;
    }
    a.fault_seed = host_mix64(fault_seed0 + (unsigned long long)it);  // fresh delay draws per iteration
    DFPR_CUDA(cudaMemsetAsync(&g->ctl.p->nheavy, 0, sizeof(long long), s));
    k_jacobi<P><<<grid, kNT, 0, s>>>(a, a.R, a.C, R2, C2, listed ? g->affected_list.p : nullptr,
                                     listed ? count : (long long)g->n, listed ? 1 : 0);
    DFPR_LAUNCHED();
    k_jacobi_heavy_scan<<<1, 1024, 0, s>>>(g->ctl.p, a.jh_rem, a.jh_off, a.jh_cap);
    DFPR_LAUNCHED();
    k_jacobi_heavy<P><<<grid, kNT, 0, s>>>(a, a.R, a.C, R2, C2, listed ? 1 : 0);
    DFPR_LAUNCHED();
    DFPR_CUDA(cudaMemcpyAsync(g->pinned, &g->ctl.p->max_change_bits, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, s));
    DFPR_CUDA(cudaMemcpyAsync(g->pinned + 1, &g->ctl.p->len.v, sizeof(long long),
                              cudaMemcpyDeviceToHost, s));
    DFPR_CUDA(cudaStreamSynchronize(s));
    memcpy(&last, &g->pinned[0], sizeof last);
    if (df && !all) count = (long long)g->pinned[1];
    // swap R <-> R2, C <-> C2
    swap_vectors<P>(g);
    std::swap(R2, a.R);
    std::swap(C2, a.C);
    if (last <= p.tol) {
      converged = true;
      ++it;
      break;
    }
  }
  DFPR_CUDA(cudaEventRecord(e1, s));
  CtlHost h = read_ctl(g);
  if (st) {
    fill_stats(h.c, st);
    st->passes = it;
    st->residual_linf = last;
    st->affected = df && !all ? count : g->n;
  }
  if (df) {
    k_clear_list<<<grid_small(count), kNT, 0, s>>>(g->affected_list.p, count, g->va_bits.p, g->rc_bits.p);
    DFPR_LAUNCHED();
  }
  return converged ? DFPR_OK : DFPR_ENOTCONV;
}

template <class P>
void normalize_ranks(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  double* sum = &g->ctl.p->dsum;
  DFPR_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), s));
  typename P::val* R;
  typename P::contrib* C;
  if constexpr (sizeof(typename P::val) == 8) {
    R = (typename P::val*)g->R64.p;
    C = (typename P::contrib*)g->C64.p;
  } else {
    R = (typename P::val*)g->R32.p;
    C = (typename P::contrib*)g->C32.p;
  }
  k_sum_ranks<typename P::val><<<grid_small(g->n), kNT, 0, s>>>(g->n, R, sum);
  DFPR_LAUNCHED();
  k_scale<typename P::val, typename P::contrib><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, R, C, sum);
  DFPR_LAUNCHED();
}

template <class P>
dfpr_status run_any(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st) {
  cudaStream_t s = g->stream;
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
  if (p.fault_crash_warps > 0) {  // checked before any device work
    const int grid = p.mode == DFPR_MODE_WORKLIST ? worklist_grid<P>(g, p)
                                                  : round_grid<P>(g, p);
    DFPR_REQUIRE((long long)p.fault_crash_warps < (long long)grid * kWPB, DFPR_EINVAL,
                 "fault_crash_warps must be below the number of warps of the launch");
  }
  if (kind == kRunStatic) reset_ranks(g);
  dfpr_status r;
  float kernel_ms = -1.f;  // set when the update ran from a captured CUDA graph
  if (p.mode == DFPR_MODE_WORKLIST) r = run_worklist<P>(g, p, kind, st, e0, e1, false, &kernel_ms);
  else if (p.mode == DFPR_MODE_ROUND) r = run_round<P>(g, p, kind, st, e0, e1);
  else r = run_jacobi<P>(g, p, kind, st, e0, e1);
  if (p.normalize && r == DFPR_OK) normalize_ranks<P>(g);
  float ms = kernel_ms;
  if (ms < 0.f) {
    DFPR_CUDA(cudaEventSynchronize(e1));
    DFPR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  if (st) {
    st->ms = ms;
    st->status = r;
  }
  // the pending change set has been consumed
  g->pend.n_src = 0;
  g->pend.n_dst = 0;
  return r;
}

}  // namespace

void alloc_iteration_state(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  if (g->cfg.precision == DFPR_FP64) {
    g->R64.reset(n, s);
    g->C64.reset(n, s);
  } else {
    g->R32.reset(n, s);
    g->C32.reset(n, s);
  }
  g->state.reset(((size_t)n + 15) / 16, s);
  DFPR_CUDA(cudaMemsetAsync(g->state.p, 0, sizeof(uint32_t) * g->state.count, s));
  unsigned long long q = 1024;
  while (q < 2ull * (unsigned long long)n) q <<= 1;
  g->qcap = q;
  g->queue.reset(q, s);
  k_fill<int32_t><<<grid_small((long long)q), kNT, 0, s>>>(g->queue.p, (long long)q, -1);
  DFPR_LAUNCHED();
  g->tcap = 1ull << 21;  // chunk tokens in flight at most (slots are reused as they drain)
  g->tokens.reset(g->tcap, s);
  k_fill<unsigned long long><<<grid_small((long long)g->tcap), kNT, 0, s>>>(g->tokens.p, (long long)g->tcap, ~0ull);
  DFPR_LAUNCHED();
  g->jcap = 4096;  // heavy vertices whose gathers can be split at the same time
  g->job_ring.reset(g->jcap, s);
  g->job_v.reset(g->jcap, s);
  g->job_rem.reset(g->jcap, s);
  g->job_sum.reset(g->jcap, s);
  g->ctl.reset(1, s);
  DFPR_CUDA(cudaMemsetAsync(g->ctl.p, 0, sizeof(DfCtl), s));
  g->affected_list.reset(n, s);
  k_fill<int32_t><<<grid_small(n), kNT, 0, s>>>(g->affected_list.p, n, -1);
  DFPR_LAUNCHED();
  g->va_bits.reset(((size_t)n + 31) / 32, s);
  g->rc_bits.reset(((size_t)n + 31) / 32, s);
  DFPR_CUDA(cudaMemsetAsync(g->va_bits.p, 0, sizeof(uint32_t) * g->va_bits.count, s));
  DFPR_CUDA(cudaMemsetAsync(g->rc_bits.p, 0, sizeof(uint32_t) * g->rc_bits.count, s));
}

void reset_ranks(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  if (g->cfg.precision == DFPR_FP64)
    k_init_ranks<double, long long><<<grid_small(g->n), kNT, 0, s>>>(
        g->n, g->out.rows.p, g->nparts > 1 ? g->part_off.p : nullptr, g->nparts, g->R64.p, g->C64.p);
  else
    k_init_ranks<float, float><<<grid_small(g->n), kNT, 0, s>>>(
        g->n, g->out.rows.p, g->nparts > 1 ? g->part_off.p : nullptr, g->nparts, g->R32.p, g->C32.p);
  DFPR_LAUNCHED();
}

double rank_sum(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  double* sum = (double*)(g->host_sync.p + 8);
  DFPR_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), s));
  if (g->cfg.precision == DFPR_FP64)
    k_sum_ranks<double><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->R64.p, sum);
  else
    k_sum_ranks<float><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->R32.p, sum);
  DFPR_LAUNCHED();
  unsigned long long bits = read_word(g, sum, sizeof(double));
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
}

double dangling_mass(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  double* sum = (double*)(g->host_sync.p + 8);
  DFPR_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), s));
  if (g->cfg.precision == DFPR_FP64)
    k_dangling<double><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, g->R64.p, sum);
  else
    k_dangling<float><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, g->R32.p, sum);
  DFPR_LAUNCHED();
  unsigned long long bits = read_word(g, sum, sizeof(double));
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
}

void residual(dfpr_graph* g, double alpha, double* linf, double* linf_rel) {
  cudaStream_t s = g->stream;
  unsigned long long* out = g->host_sync.p + 12;  // two words, cleared here
  double* dead = nullptr;
  if (g->cfg.dead_end == DFPR_TELEPORT) {
    dead = (double*)(g->host_sync.p + 14);
    DFPR_CUDA(cudaMemsetAsync(dead, 0, sizeof(double), s));
    if (g->cfg.precision == DFPR_FP64)
      k_dangling<double><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, g->R64.p, dead);
    else
      k_dangling<float><<<grid_small(g->n), kNT, 0, s>>>(g->n, g->out.rows.p, g->R32.p, dead);
    DFPR_LAUNCHED();
  }
  DFPR_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s));
  const unsigned grid = blocks_for(32ll * g->n, kNT, sm_cap(16u));
  const int32_t* poff = g->nparts > 1 ? g->part_off.p : nullptr;
  if (g->cfg.precision == DFPR_FP64)
    k_residual<double><<<grid, kNT, 0, s>>>(g->n, g->in.rows.p, g->in.edges.p, g->out.rows.p,
                                            g->R64.p, poff, g->nparts, alpha, dead, out);
  else
    k_residual<float><<<grid, kNT, 0, s>>>(g->n, g->in.rows.p, g->in.edges.p, g->out.rows.p,
                                           g->R32.p, poff, g->nparts, alpha, dead, out);
  DFPR_LAUNCHED();
  unsigned long long b[2];
  DFPR_CUDA(cudaMemcpyAsync(b, out, sizeof b, cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaStreamSynchronize(s));
  memcpy(linf, &b[0], sizeof(double));
  memcpy(linf_rel, &b[1], sizeof(double));
}

int full_worklist_grid(dfpr_graph* g, const dfpr_params& p) {
  dfpr_params q = p;
  q.grid_ctas = 0;
  return g->cfg.precision == DFPR_FP64 ? persistent_grid(g, q, (const void*)k_worklist<P64>)
                                       : persistent_grid(g, q, (const void*)k_worklist<P32>);
}

int default_worklist_grid(dfpr_graph* g, const dfpr_params& p) {
  dfpr_params q = p;
  q.grid_ctas = 0;
  return g->cfg.precision == DFPR_FP64 ? worklist_grid<P64>(g, q) : worklist_grid<P32>(g, q);
}

dfpr_status run_iteration(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st) {
  if (g->cfg.precision == DFPR_FP64) return run_any<P64>(g, p, kind, st);
  return run_any<P32>(g, p, kind, st);
}

void initial_affected(dfpr_graph* g, uint8_t* affected_dev, long long* count) {
  cudaStream_t s = g->stream;
  dfpr_params p;
  dfpr_default_params(&p);
  cudaEvent_t e0, e1;
  DFPR_CUDA(cudaEventCreate(&e0));
  DFPR_CUDA(cudaEventCreate(&e1));
  dfpr_status r;
  if (g->cfg.precision == DFPR_FP64) r = run_worklist<P64>(g, p, kRunDF, nullptr, e0, e1, true);
  else r = run_worklist<P32>(g, p, kRunDF, nullptr, e0, e1, true);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DFPR_REQUIRE(r == DFPR_OK, r, "dfpr_initial_affected: marking did not complete");
  k_export_state<<<grid_small(g->n), kNT, 0, s>>>(g->n, g->state.p,
                                                  g->relabeled ? g->perm.p : nullptr, affected_dev);
  DFPR_LAUNCHED();
  CtlHost h = read_ctl(g);
  if (count) *count = (long long)h.c.tail.v;
  // the marking pushed every affected vertex once: undo it
  reset_worklist_state(g);
}

}  // namespace dfpr
