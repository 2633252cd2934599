// Rank iterations: Dynamic Frontier, naive-dynamic and static schedules.
#pragma once
#include "common.cuh"

namespace dfpr {

enum RunKind { kRunDF = 0, kRunND = 1, kRunStatic = 2 };

// Runs one rank computation on g (see dfpr_df_pagerank / dfpr_nd_pagerank /
// dfpr_static_pagerank). Returns the status of the iteration (OK, ENOTCONV,
// ETIMEOUT); throws Fail on CUDA or argument errors.
dfpr_status run_iteration(dfpr_graph* g, const dfpr_params& p, RunKind kind, dfpr_stats* st);

// Checks parameters and runs one update (the body of dfpr_df_pagerank,
// dfpr_nd_pagerank, dfpr_static_pagerank; the caller holds the graph).
dfpr_status run_update(dfpr_graph* g, const dfpr_params* p, dfpr_stats* st, RunKind kind);

// CTAs of the worklist schedule's own grid for g, and of one full wave
// (params' grid_ctas ignored).
int default_worklist_grid(dfpr_graph* g, const dfpr_params& p);
int full_worklist_grid(dfpr_graph* g, const dfpr_params& p);

// Initial marking only: affected flags (device, n bytes) and their count.
void initial_affected(dfpr_graph* g, uint8_t* affected_dev, long long* count);

// Allocates the iteration state of g (ranks, flags, queue, control block).
void alloc_iteration_state(dfpr_graph* g);

// Sets every rank to 1/n and the contributions to R / outdeg.
void reset_ranks(dfpr_graph* g);

// FP64 sum of the ranks.
double rank_sum(dfpr_graph* g);

// FP64 sum of the ranks of dead ends (vertices without out-edges).
double dangling_mass(dfpr_graph* g);

// Largest residual of Eq. 1 over all vertices, absolute and relative to the
// vertex's rank, computed in FP64 from the stored ranks.
void residual(dfpr_graph* g, double alpha, double* linf, double* linf_rel);

}  // namespace dfpr
