// Device graph store (Sec. 3.4): CSR (out-rows) and CSC (in-rows) with
// sorted unique rows, built once from raw edges and updated in place by
// batches of deletions and insertions.
//
// Layout: each row owns a slot edges[off .. off + cap) holding deg <= cap
// sorted ids; rows that outgrow their slot move to a spare area at the end of
// the edge array (bump allocation); when the spare area runs out the whole
// direction is rebuilt with fresh slack.
#include <climits>

#include "graph.cuh"
#include "primitives.cuh"

namespace dfpr {

// Scratch slots (see common.cuh).
enum {
  kSFirst = 0, kSLast = 1, kSCap = 2, kSOff = 3,
  kSBKeys = 4, kSBTmp = 5, kSBFlag = 6, kSBPos = 7,
  kSRc = 10, kSRcT = 11, kSRcT2 = 12,
  kSHead = 13, kSGid = 14, kSDelPre = 15, kSGStart = 16, kSGOwner = 17,
  kSNewDeg = 18, kSWork = 19, kSSOff = 20, kSWOff = 21, kSDest = 22, kSNCap = 23,
  kSMerged = 24, kSDelFlag = 25, kSRbFlag = 26, kSRbPos = 27, kSRbDel = 28
};

// Device words of g->host_sync.
enum { kWErr = 0, kWRealDel = 1, kWRealIns = 2, kWOverflow = 3, kWNGroups = 4, kWS = 5, kWW = 6,
       kWMaxDeg = 7 };

namespace {

constexpr int NT = 256;

#define GRID_STRIDE(i, n)                                                    \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
       i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ unsigned long long pack2(unsigned a, unsigned b, int bits) {
  return ((unsigned long long)a << bits) | b;
}

__device__ __forceinline__ int slack_cap(int deg, double frac, int minslack) {
  long long s = (long long)((double)deg * frac);
  if (s < minslack) s = minslack;
  long long c = (long long)deg + s;
  return c > INT_MAX ? INT_MAX : (int)c;
}

// First index in a[0..len) with a[i] >= x.
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int len, int x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Last index g in [0, count) with offs[g] <= w (offs nondecreasing, offs[0] = 0).
__device__ __forceinline__ long long upper_index(const long long* offs, long long count, long long w) {
  long long lo = 0, hi = count;
  while (hi - lo > 1) {
    long long mid = (lo + hi) >> 1;
    if (offs[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            long long m, int32_t n, int bits, const int32_t* __restrict__ part_off,
                            int nparts, unsigned long long* __restrict__ keys,
                            unsigned long long* err) {
  GRID_STRIDE(i, m) {
    int a = src[i], b = dst[i];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      atomicOr(err, 1ull);
      a = 0;
      b = 0;
    } else if (nparts > 1 && part_of(part_off, nparts, a) != part_of(part_off, nparts, b)) {
      atomicOr(err, 2ull);  // an edge between two graphs of a set
      a = 0;
      b = 0;
    }
    keys[i] = pack2((unsigned)a, (unsigned)b, bits);
  }
}

__global__ void k_self_keys(int32_t n, int bits, unsigned long long* keys) {
  GRID_STRIDE(i, n) keys[i] = pack2((unsigned)i, (unsigned)i, bits);
}

__global__ void k_head_flags(const unsigned long long* __restrict__ k, long long m, uint32_t* f) {
  GRID_STRIDE(i, m) f[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void k_compact_u64(const unsigned long long* __restrict__ in,
                              const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                              long long m, unsigned long long* __restrict__ out) {
  GRID_STRIDE(i, m) if (flag[i]) out[pos[i]] = in[i];
}

__global__ void k_row_bounds(const unsigned long long* __restrict__ k, long long m, int bits,
                             long long* first, long long* last) {
  GRID_STRIDE(i, m) {
    unsigned a = (unsigned)(k[i] >> bits);
    if (i == 0 || (unsigned)(k[i - 1] >> bits) != a) first[a] = i;
    if (i == m - 1 || (unsigned)(k[i + 1] >> bits) != a) last[a] = i + 1;
  }
}

__global__ void k_caps(const long long* first, const long long* last, int32_t n, double frac,
                       int minslack, long long* cap) {
  GRID_STRIDE(u, n) cap[u] = slack_cap((int)(last[u] - first[u]), frac, minslack);
}

__global__ void k_scatter_edges(const unsigned long long* __restrict__ k, long long m, int bits,
                                const long long* __restrict__ first,
                                const long long* __restrict__ off, int32_t* __restrict__ edges) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) {
    unsigned a = (unsigned)(k[i] >> bits);
    edges[off[a] + (i - first[a])] = (int32_t)(k[i] & mask);
  }
}

__global__ void k_fill_rows(const long long* first, const long long* last, const long long* cap,
                            const long long* off, int32_t n, RowDesc* rows) {
  GRID_STRIDE(u, n) {
    RowDesc r;
    r.off = off[u];
    r.deg = (int)(last[u] - first[u]);
    r.cap = (int)cap[u];
    rows[u] = r;
  }
}

__global__ void k_transpose2(const unsigned long long* __restrict__ k, long long m, int bits,
                             unsigned long long* __restrict__ out) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) out[i] = pack2((unsigned)(k[i] & mask), (unsigned)(k[i] >> bits), bits);
}

// Batch keys: (owner << (bits + 1)) | (other << 1) | type, type 0 = deletion.
__global__ void k_batch_keys(const int32_t* ds, const int32_t* dd, long long nd, const int32_t* is,
                             const int32_t* id, long long ni, int32_t n, int bits,
                             const int32_t* __restrict__ perm, unsigned long long* keys,
                             unsigned long long* err) {
  GRID_STRIDE(i, nd + ni) {
    const bool del = i < nd;
    int a = del ? ds[i] : is[i - nd];
    int b = del ? dd[i] : id[i - nd];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      atomicOr(err, 1ull);
      a = 0;
      b = 0;
    }
    if (perm) {  // caller ids -> internal ids
      a = perm[a];
      b = perm[b];
    }
    keys[i] = ((unsigned long long)a << (bits + 1)) | ((unsigned long long)b << 1) | (del ? 0ull : 1ull);
  }
}

// Real changes: a deletion of a present edge that is not a protected self-loop
// and is not re-inserted by the same batch; an insertion of an absent edge.
__global__ void k_classify(const unsigned long long* __restrict__ uk, long long nu, int bits,
                           const RowDesc* __restrict__ rows, const int32_t* __restrict__ edges,
                           int self_loops, uint32_t* __restrict__ flag, unsigned long long* cnt) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, nu) {
    const unsigned long long key = uk[i];
    const int t = (int)(key & 1);
    const int b = (int)((key >> 1) & mask);
    const int a = (int)(key >> (bits + 1));
    const RowDesc r = rows[a];
    const int p = lower_bound_i32(edges + r.off, r.deg, b);
    const bool exists = p < r.deg && edges[r.off + p] == b;
    bool real;
    if (t == 0)
      real = exists && !(self_loops && a == b) && !(i + 1 < nu && uk[i + 1] == (key | 1ull));
    else
      real = !exists;
    flag[i] = real ? 1u : 0u;
    if (real) atomicAdd(&cnt[t], 1ull);
  }
}

__global__ void k_transpose3(const unsigned long long* __restrict__ k, long long m, int bits,
                             unsigned long long* __restrict__ out) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) {
    unsigned long long key = k[i];
    unsigned long long a = key >> (bits + 1), b = (key >> 1) & mask, t = key & 1;
    out[i] = (b << (bits + 1)) | (a << 1) | t;
  }
}

__global__ void k_seg_flags(const unsigned long long* __restrict__ rc, long long nrc, int bits,
                            uint32_t* head, uint32_t* delf) {
  GRID_STRIDE(i, nrc) {
    const unsigned long long o = rc[i] >> (bits + 1);
    head[i] = (i == 0 || (rc[i - 1] >> (bits + 1)) != o) ? 1u : 0u;
    delf[i] = (rc[i] & 1ull) ? 0u : 1u;
  }
}

__global__ void k_groups(const unsigned long long* __restrict__ rc, long long nrc, int bits,
                         const uint32_t* __restrict__ head, const uint32_t* __restrict__ gid,
                         long long* gstart, int32_t* gowner) {
  GRID_STRIDE(i, nrc) {
    if (head[i]) {
      gstart[gid[i]] = i;
      gowner[gid[i]] = (int32_t)(rc[i] >> (bits + 1));
    }
    if (i == 0) gstart[gid[nrc]] = nrc;  // gid[nrc] holds the group count
  }
}

__global__ void k_plan(long long nrc, const uint32_t* __restrict__ gid_total,
                       const long long* __restrict__ gstart, const int32_t* __restrict__ gowner,
                       const uint32_t* __restrict__ delpre, const RowDesc* __restrict__ rows,
                       double frac, int minslack, unsigned long long* tail, long long ecap,
                       long long* newdeg, long long* work, long long* dest, int32_t* ncap,
                       unsigned long long* overflow) {
  const long long ng = *gid_total;
  GRID_STRIDE(g, nrc) {
    if (g >= ng) {
      newdeg[g] = 0;
      work[g] = 0;
      continue;
    }
    const int u = gowner[g];
    const RowDesc r = rows[u];
    const long long gs = gstart[g], ge = gstart[g + 1];
    const long long nd = (long long)delpre[ge] - delpre[gs];
    const long long ni = (ge - gs) - nd;
    const long long d2 = r.deg - nd + ni;
    newdeg[g] = d2;
    work[g] = r.deg + (ge - gs);
    if (d2 <= r.cap) {
      dest[g] = r.off;
      ncap[g] = r.cap;
    } else {
      const int c = slack_cap((int)d2, frac, minslack);
      const unsigned long long p = atomicAdd(tail, (unsigned long long)c);
      if ((long long)p + c > ecap) {
        atomicOr(overflow, 1ull);
        dest[g] = -1;
      } else {
        dest[g] = (long long)p;
      }
      ncap[g] = c;
    }
  }
}

// Merge by rank: every old element and every inserted element computes its
// position in the new row from counts of smaller deleted / inserted ids.
__global__ void k_merge_flat(long long W, const uint32_t* __restrict__ gid_total,
                             const long long* __restrict__ woff, const long long* __restrict__ soff,
                             const long long* __restrict__ gstart, const int32_t* __restrict__ gowner,
                             const uint32_t* __restrict__ delpre,
                             const unsigned long long* __restrict__ rc, int bits,
                             const RowDesc* __restrict__ rows, const int32_t* __restrict__ edges,
                             int32_t* __restrict__ merged) {
  const long long ng = *gid_total;
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(w, W) {
    const long long g = upper_index(woff, ng, w);
    const long long local = w - woff[g];
    const RowDesc r = rows[gowner[g]];
    const long long gs = gstart[g], ge = gstart[g + 1];
    const int seglen = (int)(ge - gs);
    const uint32_t dbase = delpre[gs];
    if (local < r.deg) {
      const int x = edges[r.off + local];
      int lo = 0, hi = seglen;  // first segment entry with other >= x
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int)((rc[gs + mid] >> 1) & mask) < x) lo = mid + 1; else hi = mid;
      }
      if (lo < seglen && (int)((rc[gs + lo] >> 1) & mask) == x) continue;  // deleted
      const long long dels_before = (long long)delpre[gs + lo] - dbase;
      const long long ins_before = lo - dels_before;
      merged[soff[g] + local - dels_before + ins_before] = x;
    } else {
      const int j = (int)(local - r.deg);
      const unsigned long long key = rc[gs + j];
      if (!(key & 1ull)) continue;  // deletions produce nothing
      const int y = (int)((key >> 1) & mask);
      const int c = lower_bound_i32(edges + r.off, r.deg, y);
      const long long dels_before = (long long)delpre[gs + j] - dbase;
      const long long ins_before = j - dels_before;
      merged[soff[g] + c - dels_before + ins_before] = y;
    }
  }
}

__global__ void k_copy_back(long long S, const uint32_t* __restrict__ gid_total,
                            const long long* __restrict__ soff, const long long* __restrict__ dest,
                            const int32_t* __restrict__ merged, int32_t* __restrict__ edges) {
  const long long ng = *gid_total;
  GRID_STRIDE(s, S) {
    const long long g = upper_index(soff, ng, s);
    edges[dest[g] + (s - soff[g])] = merged[s];
  }
}

__global__ void k_update_rows(const uint32_t* __restrict__ gid_total, long long nrc,
                              const int32_t* __restrict__ gowner, const long long* __restrict__ dest,
                              const long long* __restrict__ newdeg, const int32_t* __restrict__ ncap,
                              RowDesc* rows) {
  const long long ng = *gid_total;
  GRID_STRIDE(g, nrc) {
    if (g >= ng) continue;
    RowDesc r;
    r.off = dest[g];
    r.deg = (int)newdeg[g];
    r.cap = ncap[g];
    rows[gowner[g]] = r;
  }
}

template <typename T, typename CT>
__global__ void k_group_contrib(const uint32_t* __restrict__ gid_total, long long nrc,
                                const int32_t* __restrict__ gowner,
                                const long long* __restrict__ newdeg, const T* __restrict__ R,
                                CT* __restrict__ C) {
  const long long ng = *gid_total;
  GRID_STRIDE(g, nrc) {
    if (g >= ng) continue;
    const int u = gowner[g];
    C[u] = contrib_of(R[u], (int)newdeg[g]);
  }
}

template <typename T, typename CT>
__global__ void k_contrib_all(int32_t n, const RowDesc* __restrict__ rows, const T* __restrict__ R,
                              CT* __restrict__ C) {
  GRID_STRIDE(u, n) C[u] = contrib_of(R[u], rows[u].deg);
}

// Appends the groups' sources and the deletion targets to the pending change
// set; cap_src / cap_dst are the room the host reserved (writes beyond are
// dropped and flagged, never performed).
__global__ void k_append_pending(const uint32_t* __restrict__ gid_total, long long nrc,
                                 const int32_t* __restrict__ gowner,
                                 const unsigned long long* __restrict__ rc, int bits,
                                 const uint32_t* __restrict__ delf, const uint32_t* __restrict__ delpre,
                                 int32_t* psrc, long long cap_src, int32_t* pdst, long long cap_dst,
                                 unsigned long long* err) {
  const long long ng = *gid_total;
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, nrc) {
    if (i < ng) {
      if (i < cap_src) psrc[i] = gowner[i];
      else atomicOr(err, 2ull);
    }
    if (delf[i]) {
      if ((long long)delpre[i] < cap_dst) pdst[delpre[i]] = (int32_t)((rc[i] >> 1) & mask);
      else atomicOr(err, 2ull);
    }
  }
}

__global__ void k_deg_of(const RowDesc* __restrict__ rows, int32_t n, long long* deg) {
  GRID_STRIDE(u, n) deg[u] = rows[u].deg;
}

// Warp per row: copies a row's ids (optionally as packed keys) to a packed array.
__global__ void k_export_rows(const RowDesc* __restrict__ rows, const int32_t* __restrict__ edges,
                              int32_t n, const long long* __restrict__ poff, int32_t* __restrict__ idx,
                              unsigned long long* __restrict__ keys, int bits) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = warp; u < n; u += nwarps) {
    const RowDesc r = rows[u];
    const long long o = poff[u];
    for (int e = lane; e < r.deg; e += 32) {
      const int x = edges[r.off + e];
      if (idx) idx[o + e] = x;
      if (keys) keys[o + e] = pack2((unsigned)u, (unsigned)x, bits);
    }
  }
}

__global__ void k_type_flags(const unsigned long long* __restrict__ rc, long long nrc, int want,
                             uint32_t* f) {
  GRID_STRIDE(i, nrc) f[i] = ((int)(rc[i] & 1ull) == want) ? 1u : 0u;
}

__global__ void k_compact_plain(const unsigned long long* __restrict__ rc, const uint32_t* flag,
                                const uint32_t* pos, long long nrc, int bits,
                                unsigned long long* out) {
  GRID_STRIDE(i, nrc) if (flag[i]) out[pos[i]] = rc[i] >> 1;  // (owner << bits) | other
}

__global__ void k_not_in(const unsigned long long* __restrict__ keys, long long m,
                         const unsigned long long* __restrict__ del, long long nd, uint32_t* keep) {
  GRID_STRIDE(i, m) {
    const unsigned long long x = keys[i];
    long long lo = 0, hi = nd;
    while (lo < hi) {
      long long mid = (lo + hi) >> 1;
      if (del[mid] < x) lo = mid + 1; else hi = mid;
    }
    keep[i] = (lo < nd && del[lo] == x) ? 0u : 1u;
  }
}

__global__ void k_degree_count(const unsigned long long* __restrict__ k, long long m, int bits,
                               uint32_t* deg) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) {
    atomicAdd(deg + (k[i] >> bits), 1u);
    atomicAdd(deg + (k[i] & mask), 1u);
  }
}

// Sort key of a vertex: decreasing degree, then increasing id. In a set of
// graphs the graph comes first (so each keeps its id range) and the degree is
// clamped to 16 bits.
__global__ void k_vertex_keys(const uint32_t* __restrict__ deg, int32_t n,
                              const int32_t* __restrict__ part_off, int nparts,
                              unsigned long long* key) {
  GRID_STRIDE(u, n) {
    if (nparts > 1) {
      const unsigned long long part = (unsigned long long)part_of(part_off, nparts, (int)u);
      const unsigned d = min(deg[u], 0xffffu);
      key[u] = (part << 48) | ((unsigned long long)(0xffffu - d) << 32) | (unsigned)u;
    } else {
      key[u] = ((unsigned long long)(0xffffffffu - deg[u]) << 32) | (unsigned)u;
    }
  }
}

__global__ void k_perm_from_sorted(const unsigned long long* __restrict__ sorted, int32_t n,
                                   int32_t* perm, int32_t* iperm) {
  GRID_STRIDE(i, n) {
    const int32_t u = (int32_t)(sorted[i] & 0xffffffffull);
    iperm[i] = u;
    perm[u] = (int32_t)i;
  }
}

__global__ void k_relabel_keys(unsigned long long* k, long long m, int bits,
                               const int32_t* __restrict__ perm) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) {
    const unsigned a = (unsigned)perm[k[i] >> bits], b = (unsigned)perm[k[i] & mask];
    k[i] = pack2(a, b, bits);
  }
}

// Packed keys (caller_row << bits | caller_col) of every edge of one direction.
__global__ void k_export_keys(const RowDesc* __restrict__ rows, const int32_t* __restrict__ edges,
                              int32_t n, const long long* __restrict__ poff,
                              const int32_t* __restrict__ iperm, int bits,
                              unsigned long long* __restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < n; i += nwarps) {
    const RowDesc r = rows[i];
    const long long o = poff[i];
    const unsigned ru = (unsigned)iperm[i];
    for (int e = lane; e < r.deg; e += 32) keys[o + e] = pack2(ru, (unsigned)iperm[edges[r.off + e]], bits);
  }
}

__global__ void k_keys_to_csr(const unsigned long long* __restrict__ k, long long m, int bits,
                              int32_t* idx, long long* first, long long* last) {
  const unsigned long long mask = (1ull << bits) - 1;
  GRID_STRIDE(i, m) {
    const unsigned a = (unsigned)(k[i] >> bits);
    idx[i] = (int32_t)(k[i] & mask);
    if (i == 0 || (unsigned)(k[i - 1] >> bits) != a) first[a] = i;
    if (i == m - 1 || (unsigned)(k[i + 1] >> bits) != a) last[a] = i + 1;
  }
}

__global__ void k_offsets_from_bounds(const long long* __restrict__ first,
                                      const long long* __restrict__ last, int32_t n,
                                      long long* deg) {
  GRID_STRIDE(u, n) deg[u] = last[u] - first[u];
}

// Largest degree over the rows of one direction, folded into *out.
__global__ void k_max_degree(const RowDesc* __restrict__ rows, int32_t n, unsigned long long* out) {
  unsigned long long d = 0;
  GRID_STRIDE(u, n) d = max(d, (unsigned long long)rows[u].deg);
  for (int k = 16; k > 0; k >>= 1) d = max(d, __shfl_down_sync(0xffffffffu, d, k));
  if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(out, d);
}

unsigned grid_for(long long n) { return blocks_for(n, NT, sm_cap(32u)); }

}  // namespace

int id_bits(int32_t n) {
  int b = 1;
  while (b < 31 && (1ll << b) < (long long)n) ++b;
  return b;
}

unsigned long long read_word(dfpr_graph* g, const void* dev_ptr, size_t bytes) {
  g->pinned[0] = 0;
  DFPR_CUDA(cudaMemcpyAsync(g->pinned, dev_ptr, bytes, cudaMemcpyDeviceToHost, g->stream));
  DFPR_CUDA(cudaStreamSynchronize(g->stream));
  return g->pinned[0];
}

namespace {

// Grows a device array keeping its first `used` elements.
template <typename T>
void grow_keep(DevArray<T>& a, long long used, long long need, cudaStream_t s) {
  if ((long long)a.count >= need) return;
  DevArray<T> b;
  b.reset((size_t)(need + need / 2 + 64), s);
  if (used > 0) DFPR_CUDA(cudaMemcpyAsync(b.p, a.p, sizeof(T) * used, cudaMemcpyDeviceToDevice, s));
  std::swap(a.p, b.p);
  std::swap(a.count, b.count);
  std::swap(a.s, b.s);
  std::swap(a.rec, b.rec);
}

// Builds one direction from sorted unique packed keys (owner << bits | other).
void build_direction(dfpr_graph* g, Rows& dir, const unsigned long long* keys, long long m) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  Scratch& sc = g->scratch;
  long long* first = sc.get<long long>(kSFirst, n, s);
  long long* last = sc.get<long long>(kSLast, n, s);
  long long* cap = sc.get<long long>(kSCap, n, s);
  long long* off = sc.get<long long>(kSOff, (size_t)n + 1, s);
  DFPR_CUDA(cudaMemsetAsync(first, 0, sizeof(long long) * n, s));
  DFPR_CUDA(cudaMemsetAsync(last, 0, sizeof(long long) * n, s));
  if (m > 0) {
    k_row_bounds<<<grid_for(m), NT, 0, s>>>(keys, m, g->bits, first, last);
    DFPR_LAUNCHED();
  }
  k_caps<<<grid_for(n), NT, 0, s>>>(first, last, n, g->cfg.row_slack, g->cfg.min_slack, cap);
  DFPR_LAUNCHED();
  scan_exclusive_i64(cap, off, n, off + n, sc, s);
  const long long total = (long long)read_word(g, off + n, sizeof(long long));
  const long long reserve = (long long)(g->cfg.tail_slack * (double)m) + 1024;
  dir.ecap = total + reserve;
  dir.edges.reset((size_t)dir.ecap, s);
  if ((long long)dir.rows.count != n) dir.rows.reset(n, s);
  if (m > 0) {
    k_scatter_edges<<<grid_for(m), NT, 0, s>>>(keys, m, g->bits, first, off, dir.edges.p);
    DFPR_LAUNCHED();
  }
  k_fill_rows<<<grid_for(n), NT, 0, s>>>(first, last, cap, off, n, dir.rows.p);
  DFPR_LAUNCHED();
  if (!dir.tail.p) dir.tail.reset(1, s);
  k_set_u64<<<1, 1, 0, s>>>(dir.tail.p, (unsigned long long)total);
  DFPR_LAUNCHED();
}

// Sorted unique keys of all edges of g in one direction, plus/minus changes.
// Rebuild path for a direction whose spare area ran out.
void rebuild_direction(dfpr_graph* g, Rows& dir, const unsigned long long* rc, long long nrc) {
  cudaStream_t s = g->stream;
  Scratch& sc = g->scratch;
  const int32_t n = g->n;
  // packed offsets of the current rows
  long long* deg = sc.get<long long>(kSCap, n, s);
  long long* poff = sc.get<long long>(kSOff, (size_t)n + 1, s);
  k_deg_of<<<grid_for(n), NT, 0, s>>>(dir.rows.p, n, deg);
  DFPR_LAUNCHED();
  scan_exclusive_i64(deg, poff, n, poff + n, sc, s);
  const long long m_cur = (long long)read_word(g, poff + n, sizeof(long long));
  uint32_t* f = sc.get<uint32_t>(kSRbFlag, (size_t)nrc + 1, s);
  uint32_t* pos = sc.get<uint32_t>(kSRbPos, (size_t)nrc + 1, s);
  // insertions (plain keys), appended after the current edges
  k_type_flags<<<grid_for(nrc), NT, 0, s>>>(rc, nrc, 1, f);
  DFPR_LAUNCHED();
  scan_exclusive_u32(f, pos, nrc, pos + nrc, sc, s);
  const long long ni = (long long)(uint32_t)read_word(g, pos + nrc, sizeof(uint32_t));
  DevArray<unsigned long long> keys, tmp;
  keys.reset((size_t)(m_cur + ni + 1), s);
  tmp.reset((size_t)(m_cur + ni + 1), s);
  k_export_rows<<<grid_for(32ll * n), NT, 0, s>>>(dir.rows.p, dir.edges.p, n, poff, nullptr,
                                                   keys.p, g->bits);
  DFPR_LAUNCHED();
  k_compact_plain<<<grid_for(nrc), NT, 0, s>>>(rc, f, pos, nrc, g->bits, keys.p + m_cur);
  DFPR_LAUNCHED();
  // deletions (plain keys, already sorted)
  k_type_flags<<<grid_for(nrc), NT, 0, s>>>(rc, nrc, 0, f);
  DFPR_LAUNCHED();
  scan_exclusive_u32(f, pos, nrc, pos + nrc, sc, s);
  const long long nd = (long long)(uint32_t)read_word(g, pos + nrc, sizeof(uint32_t));
  unsigned long long* dk = sc.get<unsigned long long>(kSRbDel, (size_t)nd + 1, s);
  k_compact_plain<<<grid_for(nrc), NT, 0, s>>>(rc, f, pos, nrc, g->bits, dk);
  DFPR_LAUNCHED();
  const long long mt = m_cur + ni;
  unsigned long long* sorted = radix_sort_u64(keys.p, tmp.p, mt, 2 * g->bits, sc, s);
  unsigned long long* other = sorted == keys.p ? tmp.p : keys.p;
  DevArray<uint32_t> keep, kpos;
  keep.reset((size_t)mt + 1, s);
  kpos.reset((size_t)mt + 1, s);
  k_not_in<<<grid_for(mt), NT, 0, s>>>(sorted, mt, dk, nd, keep.p);
  DFPR_LAUNCHED();
  scan_exclusive_u32(keep.p, kpos.p, mt, kpos.p + mt, sc, s);
  const long long m_new = (long long)(uint32_t)read_word(g, kpos.p + mt, sizeof(uint32_t));
  k_compact_u64<<<grid_for(mt), NT, 0, s>>>(sorted, keep.p, kpos.p, mt, other);
  DFPR_LAUNCHED();
  build_direction(g, dir, other, m_new);
}

// Merges one direction's real changes (packed with type bit, sorted by owner)
// into its rows. For the CSR direction also refreshes contributions of the
// changed sources and appends the pending change set.
void apply_direction(dfpr_graph* g, Rows& dir, const unsigned long long* rc, long long nrc,
                     bool csr) {
  cudaStream_t s = g->stream;
  Scratch& sc = g->scratch;
  const int bits = g->bits;
  uint32_t* head = sc.get<uint32_t>(kSHead, (size_t)nrc + 1, s);
  uint32_t* gid = sc.get<uint32_t>(kSGid, (size_t)nrc + 1, s);
  uint32_t* delf = sc.get<uint32_t>(kSDelFlag, (size_t)nrc + 1, s);
  uint32_t* delpre = sc.get<uint32_t>(kSDelPre, (size_t)nrc + 1, s);
  long long* gstart = sc.get<long long>(kSGStart, (size_t)nrc + 1, s);
  int32_t* gowner = sc.get<int32_t>(kSGOwner, (size_t)nrc + 1, s);
  long long* newdeg = sc.get<long long>(kSNewDeg, (size_t)nrc + 1, s);
  long long* work = sc.get<long long>(kSWork, (size_t)nrc + 1, s);
  long long* soff = sc.get<long long>(kSSOff, (size_t)nrc + 1, s);
  long long* woff = sc.get<long long>(kSWOff, (size_t)nrc + 1, s);
  long long* dest = sc.get<long long>(kSDest, (size_t)nrc + 1, s);
  int32_t* ncap = sc.get<int32_t>(kSNCap, (size_t)nrc + 1, s);
  unsigned long long* words = g->host_sync.p;

  const unsigned gr = grid_for(nrc);
  k_seg_flags<<<gr, NT, 0, s>>>(rc, nrc, bits, head, delf);
  DFPR_LAUNCHED();
  scan_exclusive_u32(head, gid, nrc, gid + nrc, sc, s);
  scan_exclusive_u32(delf, delpre, nrc, delpre + nrc, sc, s);
  k_groups<<<gr, NT, 0, s>>>(rc, nrc, bits, head, gid, gstart, gowner);
  DFPR_LAUNCHED();
  DFPR_CUDA(cudaMemsetAsync(words + kWOverflow, 0, sizeof(unsigned long long), s));
  k_plan<<<gr, NT, 0, s>>>(nrc, gid + nrc, gstart, gowner, delpre, dir.rows.p, g->cfg.row_slack,
                           g->cfg.min_slack, dir.tail.p, dir.ecap, newdeg, work, dest, ncap,
                           words + kWOverflow);
  DFPR_LAUNCHED();
  scan_exclusive_i64(newdeg, soff, nrc, soff + nrc, sc, s);
  scan_exclusive_i64(work, woff, nrc, woff + nrc, sc, s);
  // read back: overflow flag, group count, merged size S, work W (the group
  // count is a 4-byte word: clear the 8-byte host slot before the copy lands)
  g->pinned[1] = 0;
  DFPR_CUDA(cudaMemcpyAsync(g->pinned, words + kWOverflow, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaMemcpyAsync(g->pinned + 1, gid + nrc, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaMemcpyAsync(g->pinned + 2, soff + nrc, sizeof(long long), cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaMemcpyAsync(g->pinned + 3, woff + nrc, sizeof(long long), cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaStreamSynchronize(s));
  const bool overflow = g->pinned[0] != 0;
  const long long ngroups = (long long)(uint32_t)g->pinned[1];
  const long long S = (long long)g->pinned[2];
  const long long W = (long long)g->pinned[3];

  if (overflow) {
    rebuild_direction(g, dir, rc, nrc);
  } else {
    int32_t* merged = sc.get<int32_t>(kSMerged, (size_t)S + 1, s);
    if (W > 0) {
      k_merge_flat<<<grid_for(W), NT, 0, s>>>(W, gid + nrc, woff, soff, gstart, gowner, delpre, rc,
                                              bits, dir.rows.p, dir.edges.p, merged);
      DFPR_LAUNCHED();
    }
    if (S > 0) {
      k_copy_back<<<grid_for(S), NT, 0, s>>>(S, gid + nrc, soff, dest, merged, dir.edges.p);
      DFPR_LAUNCHED();
    }
    k_update_rows<<<gr, NT, 0, s>>>(gid + nrc, nrc, gowner, dest, newdeg, ncap, dir.rows.p);
    DFPR_LAUNCHED();
  }
  if (!csr) return;
  // contributions of the changed sources use their new out-degree
  if (g->cfg.precision == DFPR_FP64)
    k_group_contrib<double, long long><<<gr, NT, 0, s>>>(gid + nrc, nrc, gowner, newdeg, g->R64.p, g->C64.p);
  else
    k_group_contrib<float, float><<<gr, NT, 0, s>>>(gid + nrc, nrc, gowner, newdeg, g->R32.p, g->C32.p);
  DFPR_LAUNCHED();
  // pending change set: sources (marking of out-rows) and deletion targets
  const long long nd = g->last_real_del;
  grow_keep(g->pend.src, g->pend.n_src, g->pend.n_src + ngroups, s);
  grow_keep(g->pend.dst, g->pend.n_dst, g->pend.n_dst + nd, s);
  DFPR_CUDA(cudaMemsetAsync(words + kWErr, 0, sizeof(unsigned long long), s));
  k_append_pending<<<gr, NT, 0, s>>>(gid + nrc, nrc, gowner, rc, bits, delf, delpre,
                                     g->pend.src.p + g->pend.n_src,
                                     (long long)g->pend.src.count - g->pend.n_src,
                                     g->pend.dst.p + g->pend.n_dst,
                                     (long long)g->pend.dst.count - g->pend.n_dst, words + kWErr);
  DFPR_LAUNCHED();
  DFPR_REQUIRE(read_word(g, words + kWErr, 8) == 0, DFPR_ECUDA,
               "apply_batch: pending change set larger than reserved (internal error)");
  g->pend.n_src += ngroups;
  g->pend.n_dst += nd;
}

}  // namespace

void graph_build(dfpr_graph* g, const int32_t* src, const int32_t* dst, long long m_raw) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  const bool loops = g->cfg.dead_end == DFPR_SELF_LOOPS;
  const long long nk = m_raw + (loops ? n : 0);
  unsigned long long* words = g->host_sync.p;
  DevArray<unsigned long long> keys, tmp;
  keys.reset((size_t)nk + 1, s);
  tmp.reset((size_t)nk + 1, s);
  DFPR_CUDA(cudaMemsetAsync(words + kWErr, 0, sizeof(unsigned long long), s));
  if (m_raw > 0) {
    k_make_keys<<<grid_for(m_raw), NT, 0, s>>>(src, dst, m_raw, n, g->bits,
                                               g->nparts > 1 ? g->part_off.p : nullptr, g->nparts,
                                               keys.p, words + kWErr);
    DFPR_LAUNCHED();
  }
  const unsigned long long err = read_word(g, words + kWErr, 8);
  if (err & 1ull) {
    set_error("dfpr_graph_load: a vertex id is outside [0, n)");
    throw Fail{DFPR_EINVAL};
  }
  if (err & 2ull) {
    set_error("dfpr_graph_load_parts: an edge joins two graphs of the set");
    throw Fail{DFPR_EINVAL};
  }
  if (loops) {
    k_self_keys<<<grid_for(n), NT, 0, s>>>(n, g->bits, keys.p + m_raw);
    DFPR_LAUNCHED();
  }
  Scratch& sc = g->scratch;
  unsigned long long* sorted = radix_sort_u64(keys.p, tmp.p, nk, 2 * g->bits, sc, s);
  unsigned long long* other = sorted == keys.p ? tmp.p : keys.p;
  long long m = 0;
  if (nk > 0) {
    DevArray<uint32_t> flag, pos;
    flag.reset((size_t)nk + 1, s);
    pos.reset((size_t)nk + 1, s);
    k_head_flags<<<grid_for(nk), NT, 0, s>>>(sorted, nk, flag.p);
    DFPR_LAUNCHED();
    scan_exclusive_u32(flag.p, pos.p, nk, pos.p + nk, sc, s);
    k_compact_u64<<<grid_for(nk), NT, 0, s>>>(sorted, flag.p, pos.p, nk, other);
    DFPR_LAUNCHED();
    m = (long long)(uint32_t)read_word(g, pos.p + nk, sizeof(uint32_t));
  }
  if (g->cfg.reorder && n > 1) {
    // Internal numbering by decreasing total degree (ties by caller id): the
    // most frequently read ranks, contributions and flags then share sectors.
    DevArray<uint32_t> deg;
    DevArray<unsigned long long> vk, vt;
    deg.reset(n, s);
    vk.reset(n, s);
    vt.reset(n, s);
    DFPR_CUDA(cudaMemsetAsync(deg.p, 0, sizeof(uint32_t) * n, s));
    if (m > 0) {
      k_degree_count<<<grid_for(m), NT, 0, s>>>(other, m, g->bits, deg.p);
      DFPR_LAUNCHED();
    }
    k_vertex_keys<<<grid_for(n), NT, 0, s>>>(deg.p, n, g->nparts > 1 ? g->part_off.p : nullptr,
                                             g->nparts, vk.p);
    DFPR_LAUNCHED();
    unsigned long long* vs = radix_sort_u64(vk.p, vt.p, n, 64, sc, s);
    g->perm.reset(n, s);
    g->iperm.reset(n, s);
    k_perm_from_sorted<<<grid_for(n), NT, 0, s>>>(vs, n, g->perm.p, g->iperm.p);
    DFPR_LAUNCHED();
    g->relabeled = true;
    if (m > 0) {
      k_relabel_keys<<<grid_for(m), NT, 0, s>>>(other, m, g->bits, g->perm.p);
      DFPR_LAUNCHED();
      unsigned long long* rs = radix_sort_u64(other, sorted, m, 2 * g->bits, sc, s);
      if (rs != other) std::swap(sorted, other);
    }
  }
  build_direction(g, g->out, other, m);
  // CSC: transposed keys, sorted
  k_transpose2<<<grid_for(m), NT, 0, s>>>(other, m, g->bits, sorted);
  DFPR_LAUNCHED();
  unsigned long long* t_sorted = radix_sort_u64(sorted, other, m, 2 * g->bits, sc, s);
  build_direction(g, g->in, t_sorted, m);
  g->m = m;
  track_max_degree(g);
}

void graph_apply(dfpr_graph* g, const int32_t* ds, const int32_t* dd, long long nd,
                 const int32_t* is, const int32_t* id, long long ni, long long* n_applied) {
  n_applied[0] = n_applied[1] = 0;
  const long long nb = nd + ni;
  if (nb == 0) return;
  cudaStream_t s = g->stream;
  Scratch& sc = g->scratch;
  const int bits = g->bits;
  const int b3 = 2 * bits + 1;
  unsigned long long* words = g->host_sync.p;
  unsigned long long* keys = sc.get<unsigned long long>(kSBKeys, (size_t)nb + 1, s);
  unsigned long long* tmp = sc.get<unsigned long long>(kSBTmp, (size_t)nb + 1, s);
  uint32_t* flag = sc.get<uint32_t>(kSBFlag, (size_t)nb + 1, s);
  uint32_t* pos = sc.get<uint32_t>(kSBPos, (size_t)nb + 1, s);
  DFPR_CUDA(cudaMemsetAsync(words, 0, sizeof(unsigned long long) * 3, s));
  k_batch_keys<<<grid_for(nb), NT, 0, s>>>(ds, dd, nd, is, id, ni, g->n, bits,
                                           g->relabeled ? g->perm.p : nullptr, keys, words + kWErr);
  DFPR_LAUNCHED();
  if (read_word(g, words + kWErr, 8) != 0) {
    set_error("dfpr_apply_batch: a vertex id is outside [0, n)");
    throw Fail{DFPR_EINVAL};
  }
  unsigned long long* sorted = radix_sort_u64(keys, tmp, nb, b3, sc, s);
  unsigned long long* uniq = sorted == keys ? tmp : keys;
  k_head_flags<<<grid_for(nb), NT, 0, s>>>(sorted, nb, flag);
  DFPR_LAUNCHED();
  scan_exclusive_u32(flag, pos, nb, pos + nb, sc, s);
  k_compact_u64<<<grid_for(nb), NT, 0, s>>>(sorted, flag, pos, nb, uniq);
  DFPR_LAUNCHED();
  const long long nu = (long long)(uint32_t)read_word(g, pos + nb, sizeof(uint32_t));
  k_classify<<<grid_for(nu), NT, 0, s>>>(uniq, nu, bits, g->out.rows.p, g->out.edges.p,
                                         g->cfg.dead_end == DFPR_SELF_LOOPS ? 1 : 0, flag,
                                         words + kWRealDel);
  DFPR_LAUNCHED();
  scan_exclusive_u32(flag, pos, nu, pos + nu, sc, s);
  unsigned long long* rc = sc.get<unsigned long long>(kSRc, (size_t)nu + 1, s);
  k_compact_u64<<<grid_for(nu), NT, 0, s>>>(uniq, flag, pos, nu, rc);
  DFPR_LAUNCHED();
  DFPR_CUDA(cudaMemcpyAsync(g->pinned, words + kWRealDel, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
  DFPR_CUDA(cudaStreamSynchronize(s));
  n_applied[0] = (long long)g->pinned[0];
  n_applied[1] = (long long)g->pinned[1];
  g->last_real_del = n_applied[0];
  const long long nrc = n_applied[0] + n_applied[1];
  if (nrc == 0) return;
  apply_direction(g, g->out, rc, nrc, true);
  unsigned long long* rct = sc.get<unsigned long long>(kSRcT, (size_t)nrc + 1, s);
  unsigned long long* rct2 = sc.get<unsigned long long>(kSRcT2, (size_t)nrc + 1, s);
  k_transpose3<<<grid_for(nrc), NT, 0, s>>>(rc, nrc, bits, rct);
  DFPR_LAUNCHED();
  unsigned long long* rcs = radix_sort_u64(rct, rct2, nrc, b3, sc, s);
  apply_direction(g, g->in, rcs, nrc, false);
  g->m += n_applied[1] - n_applied[0];
  track_max_degree(g);
}

void graph_export(dfpr_graph* g, const Rows& dir, long long* offsets, int32_t* idx) {
  cudaStream_t s = g->stream;
  const int32_t n = g->n;
  if (g->relabeled) {
    // caller ids: every edge as a (caller row, caller column) key, sorted
    long long* deg = g->scratch.get<long long>(kSCap, n, s);
    long long* poff = g->scratch.get<long long>(kSOff, (size_t)n + 1, s);
    k_deg_of<<<grid_for(n), NT, 0, s>>>(dir.rows.p, n, deg);
    DFPR_LAUNCHED();
    scan_exclusive_i64(deg, poff, n, poff + n, g->scratch, s);
    const long long m = g->m;
    DevArray<unsigned long long> keys, tmp;
    keys.reset((size_t)m + 1, s);
    tmp.reset((size_t)m + 1, s);
    k_export_keys<<<grid_for(32ll * n), NT, 0, s>>>(dir.rows.p, dir.edges.p, n, poff, g->iperm.p,
                                                     g->bits, keys.p);
    DFPR_LAUNCHED();
    unsigned long long* sk = radix_sort_u64(keys.p, tmp.p, m, 2 * g->bits, g->scratch, s);
    long long* first = g->scratch.get<long long>(kSFirst, n, s);
    long long* last = g->scratch.get<long long>(kSLast, n, s);
    DFPR_CUDA(cudaMemsetAsync(first, 0, sizeof(long long) * n, s));
    DFPR_CUDA(cudaMemsetAsync(last, 0, sizeof(long long) * n, s));
    if (m > 0) {
      k_keys_to_csr<<<grid_for(m), NT, 0, s>>>(sk, m, g->bits, idx, first, last);
      DFPR_LAUNCHED();
    }
    k_offsets_from_bounds<<<grid_for(n), NT, 0, s>>>(first, last, n, deg);
    DFPR_LAUNCHED();
    scan_exclusive_i64(deg, offsets, n, offsets + n, g->scratch, s);
    return;
  }
  long long* deg = g->scratch.get<long long>(kSCap, n, s);
  k_deg_of<<<grid_for(n), NT, 0, s>>>(dir.rows.p, n, deg);
  DFPR_LAUNCHED();
  scan_exclusive_i64(deg, offsets, n, offsets + n, g->scratch, s);
  k_export_rows<<<grid_for(32ll * n), NT, 0, s>>>(dir.rows.p, dir.edges.p, n, offsets, idx,
                                                   nullptr, g->bits);
  DFPR_LAUNCHED();
}

void track_max_degree(dfpr_graph* g) {
  if ((long long)g->n <= kDegreeLimit) {
    g->max_degree = -1;
    return;
  }
  cudaStream_t s = g->stream;
  unsigned long long* w = g->host_sync.p + kWMaxDeg;
  DFPR_CUDA(cudaMemsetAsync(w, 0, sizeof(unsigned long long), s));
  k_max_degree<<<grid_for(g->n), NT, 0, s>>>(g->out.rows.p, g->n, w);
  DFPR_LAUNCHED();
  k_max_degree<<<grid_for(g->n), NT, 0, s>>>(g->in.rows.p, g->n, w);
  DFPR_LAUNCHED();
  g->max_degree = (long long)read_word(g, w, sizeof(unsigned long long));
}

void refresh_contributions(dfpr_graph* g) {
  cudaStream_t s = g->stream;
  if (g->cfg.precision == DFPR_FP64)
    k_contrib_all<double, long long><<<grid_for(g->n), NT, 0, s>>>(g->n, g->out.rows.p, g->R64.p, g->C64.p);
  else
    k_contrib_all<float, float><<<grid_for(g->n), NT, 0, s>>>(g->n, g->out.rows.p, g->R32.p, g->C32.p);
  DFPR_LAUNCHED();
}

}  // namespace dfpr
