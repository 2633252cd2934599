// Static PageRank over a caller-provided in-edge CSR (CSC), for callers that
// cannot allocate device memory: code that runs while another component owns
// the whole device memory budget (a framework's memory pool, an inference
// server with a fixed arena), or that must not call cudaMalloc / cudaFree
// because those calls synchronise the device and would stall other work.
//
// The entry point is a variant of the library's Jacobi iteration: instead of
// vectors it allocates per graph, it keeps its scratch (the second rank
// vector, both contribution vectors and three control words) in one
// file-scope __device__ array of fixed size. That array exists on every GPU
// that loads this library and stays allocated until the process exits, which
// is why its size is capped at kNoAllocMaxVertices vertices
// (3 * 8 MiB + 256 bytes).
//
// Vertices without out-edges (dead ends) spread their rank uniformly, as the
// library does for graphs loaded with DFPR_TELEPORT: every iteration adds
// alpha * D / n to each rank, D being the rank held by dead ends in the
// previous iterate, summed in FP64. A graph with a self-loop on every vertex
// has no dead ends, so the term is zero there.
//
// Host code cannot use the array's symbol as a device address: on the host it
// names a host-side stand-in. The device address is fetched once per device
// with cudaGetSymbolAddress (with that device current) on the first call made
// on that device. The cached address belongs to the device's current context: a
// cudaDeviceReset between calls (which also frees every other device
// allocation of the process) invalidates it. Every call shares the array and
// its previous contents: the control words are cleared before they are used,
// and calls that overlap on the GPU (two streams, two threads) race on the
// array and must not be issued.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"
#include "primitives.cuh"

namespace dfpr {
namespace {

constexpr long long kNoAllocMaxVertices = 1ll << 20;
constexpr size_t kCtlBytes = 256;
constexpr size_t kScratchBytes = kCtlBytes + 3 * sizeof(double) * (size_t)kNoAllocMaxVertices;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).
unsigned char* scratch_address(int dev) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("dfpr_static_pagerank_noalloc: cudaGetSymbolAddress failed: ") +
                cudaGetErrorString(e));
      throw Fail{DFPR_ECUDA};
    }
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  return g_scratch_ptr[dev];
}

constexpr int kNT = 256;

__global__ void k_na_init(int32_t n, const int32_t* __restrict__ outdeg, double* __restrict__ R,
                          double* __restrict__ C, double* __restrict__ dsum) {
  const double r0 = 1.0 / (double)n;
  double dead = 0.0;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (long long)gridDim.x * blockDim.x) {
    R[u] = r0;
    const int d = outdeg[u];
    C[u] = d > 0 ? r0 / (double)d : 0.0;
    if (d == 0) dead += r0;
  }
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, k);
  if ((threadIdx.x & 31) == 0 && dead > 0.0) atomicAdd(dsum, dead);
}

// One Jacobi iteration of Eq. 1, a warp per vertex: Rn[v] and Cn[v] from C,
// with the dead-end term alpha * D / n (D = *dsum, the previous iterate's
// dead-end mass); the rank of every dead end of the new iterate is added to
// *dsum_next, and the largest |Rn[v] - R[v]| goes to *max_bits (non-negative
// doubles order like their bit patterns).
__global__ void __launch_bounds__(kNT) k_na_iter(int32_t n, const long long* __restrict__ off,
                                                 const int32_t* __restrict__ idx,
                                                 const int32_t* __restrict__ outdeg, double alpha,
                                                 double base, const double* __restrict__ R,
                                                 const double* __restrict__ C,
                                                 double* __restrict__ Rn, double* __restrict__ Cn,
                                                 const double* __restrict__ dsum,
                                                 double* __restrict__ dsum_next,
                                                 unsigned long long* max_bits) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const double teleport = *dsum / (double)n;
  double local_max = 0.0, dead = 0.0;
  for (long long v = warp; v < n; v += nw) {
    double s = 0.0;
    for (long long e = off[v] + lane; e < off[v + 1]; e += 32) s += C[idx[e]];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) {
      const double r = base + alpha * (s + teleport);
      Rn[v] = r;
      const int od = outdeg[v];
      Cn[v] = od > 0 ? r / (double)od : 0.0;
      if (od == 0) dead += r;
      local_max = fmax(local_max, fabs(r - R[v]));
    }
  }
  if (lane == 0 && local_max > 0.0)
    atomicMax(max_bits, (unsigned long long)__double_as_longlong(local_max));
  if (lane == 0 && dead > 0.0) atomicAdd(dsum_next, dead);
}

}  // namespace
}  // namespace dfpr

using namespace dfpr;

extern "C" dfpr_status dfpr_static_pagerank_noalloc(int32_t n, const int64_t* in_offsets,
                                                    const int32_t* in_idx,
                                                    const int32_t* out_degree, double alpha,
                                                    double tol, int32_t max_iter, double* ranks,
                                                    int32_t* iterations, void* cuda_stream) {
  if (iterations) *iterations = 0;
  if (n <= 0 || !in_offsets || !in_idx || !out_degree || !ranks) {
    set_error("dfpr_static_pagerank_noalloc: need n > 0 and non-NULL device arrays");
    return DFPR_EINVAL;
  }
  if (n > kNoAllocMaxVertices) {
    set_error("dfpr_static_pagerank_noalloc: n = " + std::to_string(n) +
              " exceeds the fixed scratch size of " + std::to_string(kNoAllocMaxVertices) +
              " vertices");
    return DFPR_EINVAL;
  }
  if (!(alpha > 0.0 && alpha < 1.0) || !(tol > 0.0) || max_iter < 1) {
    set_error("dfpr_static_pagerank_noalloc: need 0 < alpha < 1, tol > 0, max_iter >= 1");
    return DFPR_EINVAL;
  }
  try {
    int dev = 0;
    DFPR_CUDA(cudaGetDevice(&dev));
    DFPR_REQUIRE(dev >= 0 && dev < kMaxDevices, DFPR_EINVAL, "device id out of range");
    unsigned char* base_ptr = scratch_address(dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // control words: [0] the largest change, [1] and [2] the dead-end masses
    // of the current and the next iterate (they swap every iteration)
    unsigned long long* max_bits = (unsigned long long*)base_ptr;
    double* dsum = (double*)(base_ptr + 8);
    double* dsum_next = (double*)(base_ptr + 16);
    double* C = (double*)(base_ptr + kCtlBytes);
    double* Cn = C + kNoAllocMaxVertices;
    double* Rn = Cn + kNoAllocMaxVertices;
    double* Rcur = ranks;  // the caller's buffer holds one of the two rank vectors
    double* Rnext = Rn;
    const unsigned grid = (unsigned)std::min<long long>((n + kNT / 32 - 1) / (kNT / 32), sm_cap(64u));
    DFPR_CUDA(cudaMemsetAsync(dsum, 0, sizeof(double), s));
    k_na_init<<<blocks_for(n, kNT, sm_cap(16u)), kNT, 0, s>>>(n, out_degree, Rcur, C, dsum);
    DFPR_LAUNCHED();
    const double base = (1.0 - alpha) / (double)n;
    int it = 0;
    bool converged = false;
    for (; it < max_iter;) {
      DFPR_CUDA(cudaMemsetAsync(max_bits, 0, sizeof(unsigned long long), s));
      DFPR_CUDA(cudaMemsetAsync(dsum_next, 0, sizeof(double), s));
      k_na_iter<<<grid, kNT, 0, s>>>(n, (const long long*)in_offsets, in_idx, out_degree, alpha,
                                    base, Rcur, C, Rnext, Cn, dsum, dsum_next, max_bits);
      DFPR_LAUNCHED();
      unsigned long long bits = 0;  // pageable host word: no pinned allocation
      DFPR_CUDA(cudaMemcpyAsync(&bits, max_bits, sizeof bits, cudaMemcpyDeviceToHost, s));
      DFPR_CUDA(cudaStreamSynchronize(s));
      double delta;
      memcpy(&delta, &bits, sizeof delta);
      std::swap(Rcur, Rnext);
      std::swap(C, Cn);
      std::swap(dsum, dsum_next);
      ++it;
      if (delta <= tol) {
        converged = true;
        break;
      }
    }
    if (Rcur != ranks)
      DFPR_CUDA(cudaMemcpyAsync(ranks, Rcur, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    DFPR_CUDA(cudaStreamSynchronize(s));
    if (iterations) *iterations = it;
    if (!converged) {
      set_error("dfpr_static_pagerank_noalloc: the iteration cap was reached before convergence");
      return DFPR_ENOTCONV;
    }
    return DFPR_OK;
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("dfpr_static_pagerank_noalloc: unexpected internal error");
    return DFPR_ECUDA;
  }
}
