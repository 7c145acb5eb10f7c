// A "team" is every thread of a one-cluster grid: a thread-block cluster of
// nblocks CTAs (or a single block when nblocks == 1).  Phases of a fused
// multigrid kernel are separated by the cluster barrier (a hardware barrier
// with release/acquire semantics at cluster scope, so global-memory writes
// of one phase are seen by every CTA in the next), and sums over the team
// are formed in a fixed order through distributed shared memory, so every
// thread gets the same, run-to-run reproducible value.
#pragma once
#include <cooperative_groups.h>
#include <stdint.h>

namespace hhg {

struct Team {
  unsigned nblocks;  // CTAs in the cluster; the grid is exactly one cluster

  __device__ __forceinline__ unsigned rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ unsigned size() const { return nblocks * blockDim.x; }
  __device__ __forceinline__ void sync() const {
    if (nblocks > 1)
      cooperative_groups::this_cluster().sync();
    else
      __syncthreads();
  }
};

// Sum of W values over the team.  Block partials (warp shuffles, then warps
// in order) are published in each CTA's shared memory; after the cluster
// barrier every thread adds the CTAs' partials in rank order.
template <int W>
__device__ __forceinline__ void team_sum(const Team& T, double (&v)[W]) {
  __shared__ double sh[W][33];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    double x = v[w];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[w][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double acc = 0;
      for (unsigned q = 0; q < blockDim.x / 32; ++q) acc += sh[w][q];
      sh[w][32] = acc;
    }
  }
  T.sync();
#pragma unroll
  for (int w = 0; w < W; ++w) {
    if (T.nblocks > 1) {
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      double acc = 0;
      for (unsigned r = 0; r < T.nblocks; ++r) acc += *cl.map_shared_rank(&sh[w][32], r);
      v[w] = acc;
    } else {
      v[w] = sh[w][32];
    }
  }
  T.sync();
}

__device__ __forceinline__ double team_sum1(const Team& T, double x) {
  double v[1] = {x};
  team_sum<1>(T, v);
  return v[0];
}

}  // namespace hhg
