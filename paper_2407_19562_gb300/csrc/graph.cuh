// Device graph store: build, batch update, export.
#pragma once
#include "common.cuh"

namespace dfpr {

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

// Reads one device word back to the host (synchronises the graph's stream).
unsigned long long read_word(dfpr_graph* g, const void* dev_ptr, size_t bytes);

int id_bits(int32_t n);

}  // namespace dfpr
