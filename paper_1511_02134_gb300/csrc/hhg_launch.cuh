// Launch of a one-cluster grid: nblocks CTAs forming a single thread-block
// cluster (a plain single-block launch when nblocks == 1), with programmatic
// stream serialization like every other kernel of the library.
#pragma once
#include <cuda_runtime.h>

namespace hhg {

template <class... KArgs, class... Args>
cudaError_t launch_team(void (*kernel)(KArgs...), unsigned nblocks, unsigned threads, cudaStream_t s,
                        Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = nblocks;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = nblocks > 1 ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Largest cluster size (16, else 8) at which one cluster of `kernel` with
// `threads` threads per CTA fits on the device; allows the non-portable
// size 16 on the kernel when it is used.
template <class... KArgs>
unsigned prepare_team_kernel(void (*kernel)(KArgs...), unsigned threads) {
  if (cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)kernel, &cfg) == cudaSuccess && n >= 1) return 16;
  }
  cudaGetLastError();
  return 8;
}

}  // namespace hhg
