// Colour sweeps of the Uzawa smoother (Sec. 3.3, 3.5) on shared-memory tiles
// staged by the tensor memory accelerator (TMA).
//
// One colour launch reads the whole velocity (and pressure) field, because
// every node is a neighbour of some node of the colour, but updates only a
// quarter of the nodes.  Read straight from the padded arrays, the nodes of
// one colour lie four entries apart along x, so a warp touches four times the
// bytes it uses.  Here each CTA owns a tile of TX x TY nodes in (x, y) and a
// run of kz planes in z.  One thread copies each plane of the tile with a
// one-node halo of the staged fields (u_0, u_1, u_2 and, where the update
// needs it, p) into a ring of shared-memory planes with tensor copies
// (cp.async.bulk.tensor, completion on an mbarrier per ring slot), keeping
// up to four planes in flight.  The threads then update the tile's nodes of
// the colour from shared memory.  Nodes of one colour are not coupled by the
// 15-point pattern, so the staged values are exactly those the update reads,
// and the arithmetic is the per-node body of the grid kernels
// (hhg_node_ops.cuh) over shared-memory views.
//
// Every mbarrier wait is bounded; a wait that runs out sets the error word
// (HHG_TILE_TIMEOUT), waits (bounded) for the copies the CTA has in flight and
// returns.
#include <cuda.h>

#include <string>

#include "../../include/hhg_stokes.h"
#include "hhg_kernels.h"
#include "hhg_node_ops.cuh"

namespace hhg {

namespace {

constexpr int TX = 64, TY = 8;     // tile of interior nodes; TX a multiple of 64
// The rows of the padded arrays are grouped by x mod 4 (hhg_common.h), so a
// tile row with its halo, padded x in [x0, x0 + TX + 1], is 4 runs of
// TX / 4 + 1 positions, one per residue.  The box takes BQ positions of each
// of the 4 residues (BQ = TX/4 + 1 rounded up to 16 bytes of FP32).
constexpr int BQ = 20;
constexpr int BX = 4 * BQ;         // staged entries per tile row
constexpr int BY = TY + 2;         // box height with the halo rows
constexpr int SLOTS = 4;           // ring of staged planes
constexpr int TT = (TX / 4) * TY;  // threads: one per node of the colour in a tile plane
constexpr long long WAIT_POLLS = 1 << 20;

// Staged fields: mode 0 velocity, f - B^T p at the node (u and p); 1 velocity
// with stored RU (u); 2 pressure, B u - g at the node (u and p).
template <int MODE>
__host__ __device__ constexpr int staged_fields() {
  return MODE == 1 ? 3 : 4;
}

// Bytes of one staged field-plane, rounded up to 128 for the copy destination.
template <class T>
__host__ __device__ constexpr int plane_bytes() {
  return ((BX * BY * (int)sizeof(T) + 127) / 128) * 128;
}

template <class T, int MODE>
__host__ __device__ constexpr size_t tile_smem() {
  return (size_t)SLOTS * staged_fields<MODE>() * plane_bytes<T>() + SLOTS * sizeof(uint64_t);
}

// Shared-memory view over three consecutive staged planes of one field.
// Staged row entry of padded x q: (q mod 4) BQ + (q div 4 - x0 / 4).
template <class T>
struct SNb {
  const T* pl[3];  // planes k-1, k, k+1
  int yb;          // BX * yi of the centre node's row
  int xo[3];       // row entries of padded x q-1, q, q+1
  __device__ __forceinline__ T operator()(int dx, int dy, int dz) const {
    return pl[dz + 1][yb + BX * dy + xo[dx + 1]];
  }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < WAIT_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int t, int r, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(t), "r"(r), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Issue staged plane q (node plane k0 - 1 + q, padded z = k0 + q) into its ring slot.
template <class T, int MODE>
__device__ __forceinline__ void issue_plane(const TileMaps& tm, unsigned char* sm, uint64_t* bar, int q, int x0,
                                            int y0, int k0) {
  constexpr int NF = staged_fields<MODE>();
  const int s = q % SLOTS;
  // the slot was last read through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect(&bar[s], (uint32_t)(NF * BX * BY * sizeof(T)));
#pragma unroll
  for (int f = 0; f < NF; ++f)
    tma_load_4d(sm + (size_t)(s * NF + f) * plane_bytes<T>(), &tm.m[f], x0 / 4, 0, y0, k0 + q, &bar[s]);
}

template <class T, int MODE>
__global__ void __launch_bounds__(TT) k_colour_tma(const __grid_constant__ TileMaps tm, LevelDev<T> L, int colour,
                                                   T wfac, int kz, unsigned* err) {
  pdl_enter();
  constexpr int NF = staged_fields<MODE>();
  constexpr int FS = plane_bytes<T>() / (int)sizeof(T);  // field stride within a slot, in elements
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)SLOTS * NF * plane_bytes<T>());
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * kz, k1 = min(k0 + kz, L.nz);
  const int np = k1 - k0 + 2;  // staged planes: node planes k0 - 1 .. k1
  const int t = threadIdx.x;
  const int yq = t / (TX / 4), q4 = t - yq * (TX / 4);
  const int j = y0 + yq;
  if (t == 0) {
    for (int s = 0; s < SLOTS; ++s) mbar_init(&bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0)
    for (int q = 0; q < SLOTS && q < np; ++q) issue_plane<T, MODE>(tm, sm, bar, q, x0, y0, k0);
  int issued = min(SLOTS, np), waited = 0;
  for (int k = k0; k < k1; ++k) {
    const int q = k - k0;
    // planes q, q+1, q+2 are read; wait for those not yet waited for
    bool ok = true;
    for (; waited <= q + 2; ++waited) ok = ok && mbar_wait(&bar[waited % SLOTS], (uint32_t)((waited / SLOTS) & 1));
    if (!__syncthreads_and(ok)) {
      // a copy did not complete: report, let the copies in flight land, stop
      if (t == 0) {
        atomicExch(err, (unsigned)HHG_TILE_TIMEOUT);
        for (int w = q; w < issued; ++w) mbar_wait(&bar[w % SLOTS], (uint32_t)((w / SLOTS) & 1));
      }
      __syncthreads();
      return;
    }
    const int i = x0 + 4 * q4 + ((colour - j - k) & 3);
    if (i < L.nx && j < L.ny) {
      const int64_t c = pidx(L.px, L.pxy, i, j, k);
      const int qx = i + 1, tb = x0 / 4;
      auto entry = [&](int qq) { return (qq & 3) * BQ + (qq >> 2) - tb; };
      const T* pl[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        pl[r] = reinterpret_cast<const T*>(sm + (size_t)((q + r) % SLOTS) * NF * plane_bytes<T>());
      const int yb = BX * (yq + 1), xo0 = entry(qx - 1), xo1 = entry(qx), xo2 = entry(qx + 1);
      SNb<T> u[3];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        u[d] = SNb<T>{{pl[0] + d * FS, pl[1] + d * FS, pl[2] + d * FS}, yb, {xo0, xo1, xo2}};
      const SNb<T> pv{{pl[0] + 3 * FS, pl[1] + 3 * FS, pl[2] + 3 * FS}, yb, {xo0, xo1, xo2}};
      if (MODE == 0)
        node_vel_gs_rhs_v<false>(L, c, u, pv, wfac);
      else if (MODE == 1)
        node_vel_gs_v<false>(L, c, u, wfac);
      else
        node_pres_gs_rhs_v<false>(L, c, u, pv, wfac);
    }
    __syncthreads();
    // the slot of plane q is free: stage the next plane into it
    if (t == 0 && issued < np) {
      issue_plane<T, MODE>(tm, sm, bar, issued, x0, y0, k0);
      ++issued;
    }
  }
}

template <class T, int MODE>
void launch_tile(const TileMaps& tm, const LevelDev<T>& L, int colour, T wfac, int kz, unsigned* err, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + kz - 1) / kz);
  cfg.blockDim = dim3(TT);
  cfg.dynamicSmemBytes = tile_smem<T, MODE>();
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_colour_tma<T, MODE>, tm, L, colour, wfac, kz, err);
}

template <class T, int MODE>
void allow_smem() {
  cudaFuncSetAttribute(k_colour_tma<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem<T, MODE>());
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// Tensor maps of u_0, u_1, u_2, p of a level: 4-D over the padded array
// (px / 4 positions, 4 residues, py, pz), box (BQ, 4, BY, 1), zero fill
// outside the array.
template <class T>
int make_tile_maps(const LevelDev<T>& L, TileMaps& out, std::string& err) {
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      err = "cuTensorMapEncodeTiled is not available";
      return HHG_ECUDA;
    }
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  const T* f[4] = {L.u[0], L.u[1], L.u[2], L.p};
  const cuuint64_t dims[4] = {(cuuint64_t)(L.px / 4), 4, (cuuint64_t)(L.pxy / L.px), (cuuint64_t)(L.nalloc / L.pxy)};
  const cuuint64_t strides[3] = {(cuuint64_t)(L.px / 4) * sizeof(T), (cuuint64_t)L.px * sizeof(T),
                                 (cuuint64_t)L.pxy * sizeof(T)};
  const cuuint32_t box[4] = {BQ, 4, BY, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int q = 0; q < 4; ++q) {
    if (((uintptr_t)f[q] & 15) || (strides[0] & 15) || (strides[1] & 15) || (strides[2] & 15)) {
      err = "field not aligned for tensor copies";
      return HHG_EINVAL;
    }
    const CUresult r = encode(&out.m[q], sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                              4, (void*)f[q], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      return HHG_ECUDA;
    }
  }
  return HHG_OK;
}

template <class T>
void launch_vel_colour_tile(const TileMaps& tm, const LevelDev<T>& L, int colour, int kz, unsigned* err,
                            cudaStream_t s) {
  launch_tile<T, 0>(tm, L, colour, (T)(1.0 / (6.0 * (double)L.nuh)), kz, err, s);
}

template <class T>
void launch_vel_colour_ru_tile(const TileMaps& tm, const LevelDev<T>& L, int colour, int kz, unsigned* err,
                               cudaStream_t s) {
  launch_tile<T, 1>(tm, L, colour, (T)(1.0 / (6.0 * (double)L.nuh)), kz, err, s);
}

template <class T>
void launch_pres_colour_tile(const TileMaps& tm, const LevelDev<T>& L, int colour, int kz, unsigned* err,
                             cudaStream_t s) {
  launch_tile<T, 2>(tm, L, colour, (T)((double)L.omega / (6.0 * (double)L.c)), kz, err, s);
}

void prepare_tiled() {
  allow_smem<float, 0>();
  allow_smem<float, 1>();
  allow_smem<float, 2>();
  allow_smem<double, 0>();
  allow_smem<double, 1>();
  allow_smem<double, 2>();
}

#define HHG_TILED_INST(T)                                                                                         \
  template int make_tile_maps<T>(const LevelDev<T>&, TileMaps&, std::string&);                                    \
  template void launch_vel_colour_tile<T>(const TileMaps&, const LevelDev<T>&, int, int, unsigned*, cudaStream_t); \
  template void launch_vel_colour_ru_tile<T>(const TileMaps&, const LevelDev<T>&, int, int, unsigned*,            \
                                             cudaStream_t);                                                       \
  template void launch_pres_colour_tile<T>(const TileMaps&, const LevelDev<T>&, int, int, unsigned*, cudaStream_t);
HHG_TILED_INST(float)
HHG_TILED_INST(double)
#undef HHG_TILED_INST

}  // namespace hhg
