// Coarse-grid solver kernel (Sec. 3.7): the team routine of
// hhg_coarse_block.cuh run by one thread block or one cluster.  The coarsest
// level of the paper's set-up (level 2 of the unit cube: 206 unknowns) is far
// too small to fill more than one SM, and one block needs no grid-wide
// synchronisation; coarsest levels of larger macro meshes use a cluster.
#include <mutex>
#include <string>

#include "../../include/hhg_stokes.h"
#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"
#include "hhg_launch.cuh"

namespace hhg {

namespace {
constexpr int CT = 512;  // threads per CTA of a cluster solve

template <class T>
__global__ void __launch_bounds__(CT) k_coarse_minres(CoarseSys S, LevelDev<T> L, double* scratch, CoarseParams prm,
                                                      double* info, unsigned nblocks) {
  pdl_enter();
  coarse::minres_team(Team{nblocks}, S, L, scratch, prm, info);
}

unsigned g_coarse_cluster = 8;
}  // namespace

// Launch shape of the coarse solve: small coarse systems are latency bound
// and run in one block of 128 threads (cheap barriers, one warp per CG);
// larger ones run on a cluster.
void coarse_shape(const CoarseSys& S, unsigned& nblocks, unsigned& threads) {
  if (coarse_fits_block(S)) {
    nblocks = 1;
    threads = 128;
  } else {
    nblocks = g_coarse_cluster;
    threads = CT;
  }
}

template <class T>
void launch_coarse_solve(const CoarseSys& S, const LevelDev<T>& L, double* scratch, CoarseParams prm, double* info,
                         cudaStream_t s) {
  unsigned nb, th;
  coarse_shape(S, nb, th);
  launch_team(k_coarse_minres<T>, nb, th, s, S, L, scratch, prm, info, nb);
}

template void launch_coarse_solve<double>(const CoarseSys&, const LevelDev<double>&, double*, CoarseParams, double*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(const CoarseSys&, const LevelDev<float>&, double*, CoarseParams, double*,
                                         cudaStream_t);

void prepare_coarse_solve() {
  const unsigned a = prepare_team_kernel(k_coarse_minres<double>, CT);
  const unsigned b = prepare_team_kernel(k_coarse_minres<float>, CT);
  g_coarse_cluster = a < b ? a : b;
}

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

int coarse_solve_noalloc(const CoarseSys& S, const LevelDev<double>& L, CoarseParams prm, double* info,
                         cudaStream_t s, std::string& err) {
  const int64_t need = coarse_scratch_doubles(S);
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
  coarse_shape(S, nb, th);
  e = launch_team(k_coarse_minres<double>, nb, th, s, S, L, ptr, prm, info, nb);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("coarse solve launch: ") + cudaGetErrorString(e);
    return HHG_ECUDA;
  }
  return HHG_OK;
}

}  // namespace hhg
