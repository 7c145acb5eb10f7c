// Fused coarse-levels cycle: one thread block runs the part of the V_var cycle
// (Sec. 3.5) below a small level, i.e. pre-smoothing, residual and restriction
// down to the coarsest level, the coarse MINRES solve (Sec. 3.7), then
// prolongation and post-smoothing back up, in a single launch.  The levels
// involved have at most a few thousand nodes: launched one kernel per colour
// phase they would cost a few microseconds of launch latency each for almost
// no work.  Block-wide barriers separate the phases; the per-node arithmetic
// is the one of the grid kernels (hhg_node_ops.cuh), in the same order.
#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"
#include "hhg_node_ops.cuh"

namespace hhg {

namespace {

constexpr int ST = 512;  // threads of the fused block

template <class T>
__device__ __forceinline__ void decode3(const LevelDev<T>& L, int q, int& i, int& j, int& k) {
  i = q % L.nx;
  j = (q / L.nx) % L.ny;
  k = q / (L.nx * L.ny);
}

template <class T>
__device__ void b_vel_rhs(const LevelDev<T>& L) {
  const int n = L.nx * L.ny * L.nz;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    decode3(L, q, i, j, k);
    node_vel_rhs(L, pidx(L.px, L.pxy, i, j, k));
  }
  __syncthreads();
}

template <class T>
__device__ void b_residual(const LevelDev<T>& L) {
  const int n = L.nx * L.ny * L.nz;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    decode3(L, q, i, j, k);
    node_residual(L, pidx(L.px, L.pxy, i, j, k));
  }
  __syncthreads();
}

// One colour phase: velocity (vel = true) or pressure Gauss-Seidel, with the
// right-hand side formed at each node (FP32 velocity, and pressure), or the
// velocity right-hand side read from RU (FP64).
template <class T>
__device__ void b_colour(const LevelDev<T>& L, int colour, bool vel, T w) {
  const int nq = (L.nx + 3) / 4;
  const int n = nq * L.ny * L.nz;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int t = q % nq;
    const int j = (q / nq) % L.ny;
    const int k = q / (nq * L.ny);
    const int i = ((colour - j - k) & 3) + 4 * t;
    if (i >= L.nx) continue;
    const int64_t c = pidx(L.px, L.pxy, i, j, k);
    if (vel) {
      if (sizeof(T) == 4)
        node_vel_gs_rhs(L, c, w);
      else
        node_vel_gs(L, c, w);
    } else {
      node_pres_gs_rhs(L, c, w);
    }
  }
  __syncthreads();
}

// The same step sequence as the grid path (backward colour 3 skipped: it
// would repeat the forward one exactly).
template <class T>
__device__ void b_uzawa(const LevelDev<T>& L, T inv6nuh, T omc) {
  if (sizeof(T) != 4) b_vel_rhs(L);
  for (int q = 0; q < 4; ++q) b_colour(L, q, true, inv6nuh);
  for (int q = 2; q >= 0; --q) b_colour(L, q, true, inv6nuh);
  for (int q = 0; q < 4; ++q) b_colour(L, q, false, omc);
}

template <class T>
__device__ void b_restrict(const LevelDev<T>& Lf, const LevelDev<T>& Lc) {
  const int n = Lc.nx * Lc.ny * Lc.nz;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    decode3(Lc, q, i, j, k);
    node_restrict(Lf, Lc, i, j, k);
  }
  __syncthreads();
}

template <class T>
__device__ void b_prolong(const LevelDev<T>& Lf, const LevelDev<T>& Lc) {
  const int n = Lf.nx * Lf.ny * Lf.nz;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    decode3(Lf, q, i, j, k);
    node_prolong_add(Lf, Lc, i, j, k);
  }
  __syncthreads();
}

// Coarsest level: FP64 solve; an FP32 hierarchy goes through its FP64 copy.
__device__ void b_coarse(const SmallCycle<double>& S) {
  coarse::minres_block(S.lv[0], S.scratch, S.prm, S.info);
  __syncthreads();
}

__device__ void b_coarse(const SmallCycle<float>& S) {
  const LevelDev<float>& L = S.lv[0];
  const LevelDev<double>& D = S.c64;
  for (int64_t q = threadIdx.x; q < D.nalloc; q += blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      D.f[d][q] = (double)L.f[d][q];
      D.u[d][q] = (double)L.u[d][q];
    }
    D.g[q] = (double)L.g[q];
    D.p[q] = (double)L.p[q];
  }
  __syncthreads();
  coarse::minres_block(D, S.scratch, S.prm, S.info);
  __syncthreads();
  for (int64_t q = threadIdx.x; q < D.nalloc; q += blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][q] = (float)D.u[d][q];
    L.p[q] = (float)D.p[q];
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(ST) k_small_cycle(SmallCycle<T> S) {
  const int top = S.nlev - 1;
  for (int l = top; l >= 1; --l) {
    for (int s = 0; s < S.nu_pre[l]; ++s) b_uzawa(S.lv[l], S.inv6nuh[l], S.omc[l]);
    b_residual(S.lv[l]);
    b_restrict(S.lv[l], S.lv[l - 1]);
  }
  b_coarse(S);
  for (int l = 1; l <= top; ++l) {
    b_prolong(S.lv[l], S.lv[l - 1]);
    for (int s = 0; s < S.nu_post[l]; ++s) b_uzawa(S.lv[l], S.inv6nuh[l], S.omc[l]);
  }
}

}  // namespace

template <class T>
void launch_small_cycle(const SmallCycle<T>& S, cudaStream_t s) {
  k_small_cycle<T><<<1, ST, 0, s>>>(S);
}

template void launch_small_cycle<double>(const SmallCycle<double>&, cudaStream_t);
template void launch_small_cycle<float>(const SmallCycle<float>&, cudaStream_t);

}  // namespace hhg
