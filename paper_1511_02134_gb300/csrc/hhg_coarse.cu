// Coarse-grid solver kernel (Sec. 3.7): the block routine of
// hhg_coarse_block.cuh run by one thread block.  The coarsest level of the
// paper's set-up (level 2 of the unit cube: 206 unknowns) is far too small to
// fill more than one SM, and one block needs no grid-wide synchronisation.
#include <mutex>
#include <string>

#include "../../include/hhg_stokes.h"
#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"
#include "hhg_launch.cuh"

namespace hhg {

namespace {
constexpr int CT = 512;  // threads of the coarse block

__global__ void __launch_bounds__(CT) k_coarse_minres(LevelDev<double> L, double* scratch, CoarseParams prm,
                                                      double* info, unsigned nblocks) {
  pdl_enter();
  coarse::minres_team(Team{nblocks}, L, scratch, prm, info);
}

unsigned g_coarse_cluster = 8;
}  // namespace

// Launch shape of the coarse solve: small levels are latency bound and run in
// one block of 128 threads (cheap barriers, one warp per CG); larger ones run
// on a cluster.
void coarse_shape(const LevelDev<double>& L, unsigned& nblocks, unsigned& threads) {
  if (L.nalloc <= 2048) {
    nblocks = 1;
    threads = 128;
  } else {
    nblocks = g_coarse_cluster;
    threads = CT;
  }
}

void launch_coarse_solve(const LevelDev<double>& L, double* scratch, CoarseParams prm, double* info, cudaStream_t s) {
  unsigned nb, th;
  coarse_shape(L, nb, th);
  launch_team(k_coarse_minres, nb, th, s, L, scratch, prm, info, nb);
}

void prepare_coarse_solve() { g_coarse_cluster = prepare_team_kernel(k_coarse_minres, CT); }

// ---- allocation-free variant -------------------------------------------------
// Scratch of the coarse solve for callers that may not allocate device memory:
// a file-scope device array of NOALLOC_COARSE_DOUBLES doubles (2 MiB), which
// every GPU that loads the library holds until the process exits.  In host
// code the symbol names a host-side stand-in, so the kernel is given the
// device address looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_coarse_scratch[NOALLOC_COARSE_DOUBLES];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

int coarse_solve_noalloc(const LevelDev<double>& L, CoarseParams prm, double* info, cudaStream_t s,
                         std::string& err) {
  const int64_t need = (int64_t)COARSE_FIELDS * L.nalloc;
  if (need > NOALLOC_COARSE_DOUBLES) {
    err = "coarsest level needs " + std::to_string(need) + " scratch doubles; the allocation-free coarse solve holds " +
          std::to_string(NOALLOC_COARSE_DOUBLES);
    return HHG_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return HHG_ECUDA;
  }
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    err = "device index beyond the allocation-free table";
    return HHG_EINVAL;
  }
  double* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // once per device, with that device current (set by the caller)
      e = cudaGetSymbolAddress((void**)&g_noalloc_ptr[dev], g_noalloc_coarse_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return HHG_ECUDA;
      }
    }
    ptr = g_noalloc_ptr[dev];
  }
  unsigned nb, th;
  coarse_shape(L, nb, th);
  e = launch_team(k_coarse_minres, nb, th, s, L, ptr, prm, info, nb);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("coarse solve launch: ") + cudaGetErrorString(e);
    return HHG_ECUDA;
  }
  return HHG_OK;
}

}  // namespace hhg
