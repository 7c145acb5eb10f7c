// Fused coarse-levels cycle: one thread-block cluster (a "team",
// hhg_team.cuh) runs the part of the V_var cycle (Sec. 3.5) below a
// mid-sized level, i.e. pre-smoothing, residual and restriction down to the
// coarsest level, the coarse MINRES solve (Sec. 3.7), then prolongation and
// post-smoothing back up, in a single launch.  Launched one kernel per colour
// phase these levels cost a few microseconds of launch latency each for
// little work; here a hardware cluster barrier separates the phases.  The
// per-node arithmetic is the one of the grid kernels (hhg_node_ops.cuh), in
// the same order.
#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"
#include "hhg_launch.cuh"
#include "hhg_node_ops.cuh"
#include "hhg_team.cuh"

namespace hhg {

namespace {

constexpr int ST = 512;  // threads per CTA of the fused team

template <class T>
__device__ __forceinline__ void decode3(const LevelDev<T>& L, int q, int& i, int& j, int& k) {
  i = q % L.nx;
  j = (q / L.nx) % L.ny;
  k = q / (L.nx * L.ny);
}

template <class T>
__device__ void b_vel_rhs(const Team& tm, const LevelDev<T>& L) {
  const int n = L.nx * L.ny * L.nz;
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    int i, j, k;
    decode3(L, q, i, j, k);
    node_vel_rhs(L, node_at(L.px, L.pxy, i, j, k));
  }
  tm.sync();
}

template <class T>
__device__ void b_residual(const Team& tm, const LevelDev<T>& L) {
  const int n = L.nx * L.ny * L.nz;
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    int i, j, k;
    decode3(L, q, i, j, k);
    node_residual(L, node_at(L.px, L.pxy, i, j, k));
  }
  tm.sync();
}

// One colour phase: velocity Gauss-Seidel (what = 0), pressure Gauss-Seidel
// (what = 1), or both at each node of the colour (what = 2: the last
// velocity colour of a step with the first pressure colour), with the
// right-hand side formed at each node (FP32 velocity, and pressure), or the
// velocity right-hand side read from RU (FP64).
template <class T>
__device__ void b_colour(const Team& tm, const LevelDev<T>& L, int colour, int what, T inv6nuh, T omc) {
  const int nq = (L.nx + 3) / 4;
  const int n = nq * L.ny * L.nz;
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    const int t = q % nq;
    const int j = (q / nq) % L.ny;
    const int k = q / (nq * L.ny);
    const int i = ((colour - j - k) & 3) + 4 * t;
    if (i >= L.nx) continue;
    const Node c = node_at(L.px, L.pxy, i, j, k);
    if (what != 1) {
      if (sizeof(T) == 4)
        node_vel_gs_rhs<true>(L, c, inv6nuh);
      else
        node_vel_gs<true>(L, c, inv6nuh);
    }
    if (what != 0) node_pres_gs_rhs<true>(L, c, omc);
  }
  tm.sync();
}

// The same step sequence as the grid path (backward colour 3 skipped: it
// would repeat the forward one exactly; backward colour 0 shares its phase
// with pressure colour 0).
template <class T>
__device__ void b_uzawa(const Team& tm, const LevelDev<T>& L, T inv6nuh, T omc) {
  if (sizeof(T) != 4) b_vel_rhs(tm, L);
  for (int q = 0; q < 4; ++q) b_colour(tm, L, q, 0, inv6nuh, omc);
  for (int q = 2; q >= 1; --q) b_colour(tm, L, q, 0, inv6nuh, omc);
  b_colour(tm, L, 0, 2, inv6nuh, omc);
  for (int q = 1; q < 4; ++q) b_colour(tm, L, q, 1, inv6nuh, omc);
}

template <class T>
__device__ void b_restrict(const Team& tm, const LevelDev<T>& Lf, const LevelDev<T>& Lc) {
  const int n = Lc.nx * Lc.ny * Lc.nz;
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    int i, j, k;
    decode3(Lc, q, i, j, k);
    node_restrict(Lf, Lc, i, j, k);
  }
  tm.sync();
}

template <class T>
__device__ void b_prolong(const Team& tm, const LevelDev<T>& Lf, const LevelDev<T>& Lc) {
  const int n = Lf.nx * Lf.ny * Lf.nz;
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    int i, j, k;
    decode3(Lf, q, i, j, k);
    node_prolong_add(Lf, Lc, i, j, k);
  }
  tm.sync();
}

// Coarsest level: the FP64 coarse solve on the compact unknowns, reading and
// updating the level's fields in their own precision.  A coarse system that
// fits one block runs on the first CTA alone: its sums then need no cluster
// barrier and its three CG solves run on one warp each.
template <class T>
__device__ void b_coarse(const Team& tm, const SmallCycle<T>& S) {
  if (tm.nblocks > 1 && coarse_fits_block(S.cs)) {
    if (blockIdx.x == 0) coarse::minres_team(Team{1}, S.cs, S.lv[0], S.scratch, S.prm, S.info);
  } else {
    coarse::minres_team(tm, S.cs, S.lv[0], S.scratch, S.prm, S.info);
  }
  tm.sync();
}

template <class R>
__global__ void __launch_bounds__(ST) k_small_cycle(SmallCycle<R> S) {
  pdl_enter();
  const Team tm{S.nblocks};
  const int top = S.nlev - 1;
  for (int l = top; l >= 1; --l) {
    for (int s = 0; s < S.nu_pre[l]; ++s) b_uzawa(tm, S.lv[l], S.inv6nuh[l], S.omc[l]);
    b_residual(tm, S.lv[l]);
    b_restrict(tm, S.lv[l], S.lv[l - 1]);
  }
  b_coarse(tm, S);
  for (int l = 1; l <= top; ++l) {
    b_prolong(tm, S.lv[l], S.lv[l - 1]);
    for (int s = 0; s < S.nu_post[l]; ++s) b_uzawa(tm, S.lv[l], S.inv6nuh[l], S.omc[l]);
  }
}

}  // namespace

template <class R>
void launch_small_cycle(const SmallCycle<R>& S, cudaStream_t s) {
  launch_team(k_small_cycle<R>, S.nblocks, ST, s, S);
}

unsigned prepare_small_cycle() {
  const unsigned a = prepare_team_kernel(k_small_cycle<float>, ST);
  const unsigned b = prepare_team_kernel(k_small_cycle<double>, ST);
  return a < b ? a : b;
}

template void launch_small_cycle<double>(const SmallCycle<double>&, cudaStream_t);
template void launch_small_cycle<float>(const SmallCycle<float>&, cudaStream_t);

}  // namespace hhg
