// Device graph store: build, batch update, export.
#pragma once
#include "common.cuh"

namespace dfpr {

// Size limits. Edge keys are counted and placed with 32-bit prefix sums, so a
// graph holds at most 2^32 - 2 edges, self-loops included. A warp sums the
// degrees of the 32 rows it holds in 32-bit integers, so the update kernels
// need every in- and out-degree at most 2^25 - 1; degrees are tracked (and
// checked before an update) only when n exceeds that bound, since a degree
// never exceeds n.
constexpr long long kEdgeLimit = (1ll << 32) - 2;
constexpr long long kDegreeLimit = (1ll << 25) - 1;

// Builds CSR and CSC of g from m raw device edges (ids checked; EINVAL on a bad id).
void graph_build(dfpr_graph* g, const int32_t* src, const int32_t* dst, long long m_raw);

// Applies a batch (device arrays). Fills n_applied[0..1] = {real deletions, real insertions}
// and appends the real changes to the pending change set.
void graph_apply(dfpr_graph* g, const int32_t* del_src, const int32_t* del_dst, long long n_del,
                 const int32_t* ins_src, const int32_t* ins_dst, long long n_ins,
                 long long* n_applied);

// Packed copy of one direction: offsets[n + 1], idx[m] (device pointers).
void graph_export(dfpr_graph* g, const Rows& dir, long long* offsets, int32_t* idx);

// Recomputes the contribution array C = R / outdeg for every vertex.
void refresh_contributions(dfpr_graph* g);

// Largest in- or out-degree of g into g->max_degree when n > kDegreeLimit
// (else -1: every degree is at most n).
void track_max_degree(dfpr_graph* g);

// Reads one device word back to the host (synchronises the graph's stream).
unsigned long long read_word(dfpr_graph* g, const void* dev_ptr, size_t bytes);

int id_bits(int32_t n);

}  // namespace dfpr
