// Coarse-grid solver kernel (Sec. 3.7): the block routine of
// hhg_coarse_block.cuh run by one thread block.  The coarsest level of the
// paper's set-up (level 2 of the unit cube: 206 unknowns) is far too small to
// fill more than one SM, and one block needs no grid-wide synchronisation.
#include <mutex>
#include <string>

#include "../../include/hhg_stokes.h"
#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"

namespace hhg {

namespace {
constexpr int CT = 512;  // threads of the coarse block

__global__ void __launch_bounds__(CT) k_coarse_minres(LevelDev<double> L, double* scratch, CoarseParams prm,
                                                      double* info) {
  coarse::minres_block(L, scratch, prm, info);
}
}  // namespace

// Threads of the coarse block: small levels are latency bound, and fewer
// warps make each block-wide barrier and reduction cheaper.
int coarse_threads(const LevelDev<double>& L) { return L.nalloc <= 4096 ? 128 : CT; }

void launch_coarse_solve(const LevelDev<double>& L, double* scratch, CoarseParams prm, double* info, cudaStream_t s) {
  k_coarse_minres<<<1, coarse_threads(L), 0, s>>>(L, scratch, prm, info);
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
  k_coarse_minres<<<1, coarse_threads(L), 0, s>>>(L, ptr, prm, info);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("coarse solve launch: ") + cudaGetErrorString(e);
    return HHG_ECUDA;
  }
  return HHG_OK;
}

}  // namespace hhg
