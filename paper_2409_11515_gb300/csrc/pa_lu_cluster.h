// pa_lu_cluster.h -- Algorithm 2 (the LU route) on one thread-block cluster
// with the solve vector in distributed shared memory (pa_lu_cluster.cu).
#pragma once

#include <vector>

#include "pa_internal.h"

namespace pa {

// One triangular system in the cluster kernel's form, built by lc_build from
// the single-CTA step form (TriHost) for a cluster of C = 2^lgC CTAs.  CTA b
// owns the rows i with i mod C = b and, in step l, applies exactly the items
// of its own rows.  Its steps are one contiguous run of 16-byte records in
// `stream`: per step a block of a header {count | log2 lanes << 27,
// entries, 0, 0}, the items and the entries of their longer segments.  An
// item is {row, column, value as two words} or {~row, first, end, 0} with
// the segment's entries at block positions [first, end); an entry is
// {column, 0, value as two words}; values are -T_ij / T_ii.  A row's last
// item carries a mark (bit 30 of the row of a one-entry item, w = 1 for a
// segment); rows without items are marked in fin0.  The stream is
// cut into batches of consecutive steps of at most `cap` records (a longer
// block is a batch of its own): batch[bbase[b] .. bbase[b + 1]) holds
// {first step, end step, stream offset, records}.
struct LcSys {
  int32_t nproc;
  const int4* stream;
  const int4* batch;
  const int32_t* bbase;  // [C + 1]
  const uint8_t* fin0;   // [n] 1: the row has no items (final from the start)
  const double* dinv;    // [n] 1 / T_ii
};
struct LcHost {
  int32_t nproc = 0;
  std::vector<int4> stream, batch;
  std::vector<int32_t> bbase;
  std::vector<uint8_t> fin0;
};
constexpr int32_t kLcLast = 1 << 30;  // mark of a row's last one-entry item
// The cluster form of t (whose items and entries follow tri_analyse), in
// batches of at most cap records.
void lc_build(const TriHost& t, int lgC, int cap, LcHost* out);

// From this many rows on, engine AUTO runs the LU route on a cluster even
// where the solve vector fits one CTA's shared memory (GB300, ms per
// iteration, one CTA against the cluster: 5,766 rows 1.93 / 2.27, 10,086
// rows 3.70 / 3.34, 19,494 rows 11.2 / 4.9).
constexpr int kLuClusterMinRows = 8192;

struct LuClusterParams {
  LuGridParams g;  // vectors, reductions and run state (g.sys and g.y unused)
  LcSys sys[4];    // L, U, U^T, L^T
};

// A cluster of 2^lgC CTAs, R vector slots per CTA, staging slots of cap
// records each, and fin = 1 when each CTA also holds its rows' final values
// (steps then end without memory ordering; readers wait for the values).
struct LcPlan {
  int lgC = 0, R = 0, cap = 0, fin = 0;
};
// The plan for factors of n rows: clusters of 16 CTAs, else 8, the largest
// staging slots that fit next to the vectors, final values where they fit;
// false when the vector does not fit the cluster's shared memory or no such
// cluster can be placed on this GPU.
bool lu_cluster_plan(int n, LcPlan* plan);
// One run (g.partials: [C][4]).
cudaError_t launch_lu_cluster(const LuClusterParams& p, const LcPlan& plan, cudaStream_t s,
                              int64_t* launches);

}  // namespace pa
