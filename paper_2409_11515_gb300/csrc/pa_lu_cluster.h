// pa_lu_cluster.h -- Algorithm 2 (the LU route) on one thread-block cluster
// with the solve vector in distributed shared memory (pa_lu_cluster.cu).
#pragma once

#include "pa_internal.h"

namespace pa {

// The run's parameters: the grid kernel's, with the four systems in the
// step form of the single-CTA kernel (L, U, U^T, L^T).
struct LuClusterParams {
  LuGridParams g;
  TriSys sys[4];
};

// The cluster size (16, else 8) and per-CTA slot count R for factors of n
// rows, or 0 when the solve vector does not fit the cluster's shared memory
// or no such cluster can be placed on this GPU.
int lu_cluster_plan(int n, int* lgC, int* R);
// One run (partials: [C][4]).
cudaError_t launch_lu_cluster(const LuClusterParams& p, int lgC, int R, cudaStream_t s,
                              int64_t* launches);

}  // namespace pa
