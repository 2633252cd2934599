// Device-wide scan and sort used by the graph build and batch update.
#pragma once
#include "common.cuh"

namespace dfpr {

// Exclusive prefix sum of n values (in-place allowed). When total != nullptr
// the sum of all n values is written to *total (device memory).
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* total,
                        Scratch& sc, cudaStream_t s);
void scan_exclusive_i64(const long long* in, long long* out, long long n, long long* total,
                        Scratch& sc, cudaStream_t s);

// Sorts n keys ascending on their low `bits` bits (higher bits must be zero).
// Uses tmp (n keys) as the ping-pong buffer; returns the buffer that holds the
// sorted keys (keys or tmp).
unsigned long long* radix_sort_u64(unsigned long long* keys, unsigned long long* tmp, long long n,
                                   int bits, Scratch& sc, cudaStream_t s);

// Scratch slots reserved by the primitives (callers use 0..7).
constexpr int kSlotSortCounts = 8;
constexpr int kSlotScanSums = 9;

inline unsigned blocks_for(long long n, int per_block, unsigned cap = 1u << 30) {
  long long b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

// Multiprocessors of the current device (queried once per device and cached;
// 1 when the query fails, so that a grid cap never becomes 0).
int device_sms();

// Grid-stride cap of `per_sm` CTAs on every multiprocessor of the current device.
inline unsigned sm_cap(unsigned per_sm) { return (unsigned)device_sms() * per_sm; }

}  // namespace dfpr
