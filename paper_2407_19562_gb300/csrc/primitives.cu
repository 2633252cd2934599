// Device-wide exclusive scan and LSD radix sort (8-bit digits, stable).
#include "primitives.cuh"

namespace dfpr {

int device_sms() {
  static std::atomic<int> cache[64];  // 0 = not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}


namespace {

constexpr int kNT = 256;   // threads per block
constexpr int kIPT = 8;    // items per thread
constexpr int kTile = kNT * kIPT;

// ---------------------------------------------------------------------------
// Scan: tile-local scan, recursive scan of tile sums, add-back.
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kNT) k_scan_tile(const T* __restrict__ in, T* __restrict__ out,
                                                   T* __restrict__ sums, long long n) {
  __shared__ T tile[kTile];
  __shared__ T wsum[kNT / 32];
  const long long base = (long long)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kNT) {
    long long g = base + i;
    tile[i] = g < n ? in[g] : T(0);
  }
  __syncthreads();
  T v[kIPT];
  T acc = 0;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    v[j] = tile[threadIdx.x * kIPT + j];
    acc += v[j];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = acc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < kNT / 32 ? wsum[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < kNT / 32) wsum[lane] = t;
  }
  __syncthreads();
  T prefix = (w > 0 ? wsum[w - 1] : T(0)) + x - acc;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    tile[threadIdx.x * kIPT + j] = prefix;
    prefix += v[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTile; i += kNT) {
    long long g = base + i;
    if (g < n) out[g] = tile[i];
  }
  if (threadIdx.x == 0 && sums) sums[blockIdx.x] = wsum[kNT / 32 - 1];
}

template <typename T>
__global__ void __launch_bounds__(kNT) k_scan_add(T* __restrict__ out, const T* __restrict__ offs,
                                                  long long n) {
  const long long base = (long long)blockIdx.x * kTile;
  const T o = offs[blockIdx.x];
  for (int i = threadIdx.x; i < kTile; i += kNT) {
    long long g = base + i;
    if (g < n) out[g] += o;
  }
}

template <typename T>
void scan_rec(const T* in, T* out, long long n, T* total, T* level_buf, cudaStream_t s) {
  const long long nb = (n + kTile - 1) / kTile;
  if (nb <= 1) {
    k_scan_tile<T><<<1, kNT, 0, s>>>(in, out, total, n);
    DFPR_LAUNCHED();
    return;
  }
  T* sums = level_buf;
  k_scan_tile<T><<<(unsigned)nb, kNT, 0, s>>>(in, out, sums, n);
  DFPR_LAUNCHED();
  scan_rec<T>(sums, sums, nb, total, level_buf + nb + 1, s);
  k_scan_add<T><<<(unsigned)nb, kNT, 0, s>>>(out, sums, n);
  DFPR_LAUNCHED();
}

template <typename T>
void scan_any(const T* in, T* out, long long n, T* total, Scratch& sc, cudaStream_t s) {
  if (n <= 0) {
    if (total) DFPR_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return;
  }
  long long need = 16;
  for (long long k = n; k > 1; k = (k + kTile - 1) / kTile) need += (k + kTile - 1) / kTile + 1;
  T* lv = sc.get<T>(kSlotScanSums, (size_t)need, s);
  scan_rec<T>(in, out, n, total, lv, s);
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kNT) k_rs_hist(const unsigned long long* __restrict__ keys,
                                                 long long n, int shift,
                                                 uint32_t* __restrict__ counts, long long nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    long long i = base + (long long)j * kNT + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(long long)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: each warp ranks its 256 keys in index order with
// match-any groups; warps are then ordered by a per-digit prefix.
__global__ void __launch_bounds__(kNT) k_rs_scatter(const unsigned long long* __restrict__ in,
                                                    unsigned long long* __restrict__ out,
                                                    long long n, int shift,
                                                    const uint32_t* __restrict__ offsets,
                                                    long long nb) {
  __shared__ uint32_t wcnt[kNT / 32][256];
  __shared__ uint32_t base_off[256];
  for (int i = threadIdx.x; i < (kNT / 32) * 256; i += kNT) (&wcnt[0][0])[i] = 0;
  base_off[threadIdx.x] = offsets[(long long)threadIdx.x * nb + blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long wbase = (long long)blockIdx.x * kTile + (long long)w * 32 * kIPT;
  unsigned long long k[kIPT];
  uint32_t rank[kIPT];
  int dig[kIPT];
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const long long i = wbase + j * 32 + lane;
    const bool valid = i < n;
    k[j] = valid ? in[i] : 0ull;
    const int d = valid ? (int)((unsigned)(k[j] >> shift) & 255u) : 256 + lane;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    const unsigned peers = __match_any_sync(0xffffffffu, d) & act;
    const unsigned lower = peers & ((1u << lane) - 1u);
    uint32_t before = 0;
    if (valid) before = wcnt[w][d];
    __syncwarp();
    if (valid && lower == 0) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[j] = before + __popc(lower);
    dig[j] = d;
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    uint32_t acc = 0;
#pragma unroll
    for (int ww = 0; ww < kNT / 32; ++ww) {
      uint32_t c = wcnt[ww][d];
      wcnt[ww][d] = acc;
      acc += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const long long i = wbase + j * 32 + lane;
    if (i < n) {
      const int d = dig[j];
      out[(long long)base_off[d] + wcnt[w][d] + rank[j]] = k[j];
    }
  }
}

// One block sorts up to 2048 keys with a bitonic network in shared memory.
constexpr int kSmallSort = 2048;
__global__ void __launch_bounds__(1024) k_sort_small(unsigned long long* keys, long long n) {
  __shared__ unsigned long long s[kSmallSort];
  for (int i = threadIdx.x; i < kSmallSort; i += 1024) s[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= kSmallSort; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kSmallSort; i += 1024) {
        int p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          unsigned long long a = s[i], b = s[p];
          if ((a > b) == up) {
            s[i] = b;
            s[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += 1024) keys[i] = s[i];
}

}  // namespace

void scan_exclusive_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* total,
                        Scratch& sc, cudaStream_t s) {
  scan_any<uint32_t>(in, out, n, total, sc, s);
}

void scan_exclusive_i64(const long long* in, long long* out, long long n, long long* total,
                        Scratch& sc, cudaStream_t s) {
  scan_any<long long>(in, out, n, total, sc, s);
}

unsigned long long* radix_sort_u64(unsigned long long* keys, unsigned long long* tmp, long long n,
                                   int bits, Scratch& sc, cudaStream_t s) {
  if (n <= 1) return keys;
  if (n <= kSmallSort) {
    k_sort_small<<<1, 1024, 0, s>>>(keys, n);
    DFPR_LAUNCHED();
    return keys;
  }
  const long long nb = (n + kTile - 1) / kTile;
  DFPR_REQUIRE(nb * 256 < (1ll << 32), DFPR_EINVAL, "radix_sort_u64: too many keys");
  uint32_t* counts = sc.get<uint32_t>(kSlotSortCounts, (size_t)(nb * 256), s);
  unsigned long long* a = keys;
  unsigned long long* b = tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)nb, kNT, 0, s>>>(a, n, shift, counts, nb);
    DFPR_LAUNCHED();
    scan_exclusive_u32(counts, counts, nb * 256, nullptr, sc, s);
    k_rs_scatter<<<(unsigned)nb, kNT, 0, s>>>(a, b, n, shift, counts, nb);
    DFPR_LAUNCHED();
    unsigned long long* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace dfpr
