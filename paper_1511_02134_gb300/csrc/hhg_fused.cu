// The FP32 inexact Uzawa step (Sec. 3.3) as three colour-fused passes over a
// level, each reading the fields about once instead of once per colour.
//
// The step is the colour sequence (Sec. 3.4-3.5, colours c = (i + j + k) mod 4)
//   velocity 0 1 2 3 | velocity 2 1, velocity 0 + pressure 0 | pressure 1 2 3
// (the backward velocity colour 3 repeats the forward one exactly and is
// skipped; a colour-0 node's pressure update right after its velocity update
// keeps the sequential order, see k_vel_pres_colour0).  A pass runs F of
// these colour phases (F = 4, 3, 3) in one launch.  Each CTA owns a tile of
// 64 x Ty nodes in (x, y) and marches through the planes in z; at march step
// s, phase q updates its colour's nodes on plane s - q.  Phase q on plane k
// then reads plane k + 1 after phase q - 1 (done earlier in the same step)
// and plane k - 1 after phase q (done one step before) but before phase q + 1
// (done later in this step): exactly the values of the sequential order.
// In (x, y) the tile carries a halo of F nodes: phase q is evaluated on the
// tile widened by F - 1 - q, so the last phase is exact on the tile itself.
// The halo nodes' values are provisional copies of the neighbouring tiles'
// and are never written back.
//
// Staging: the input fields (u_0, u_1, u_2, p) of each plane of the widened
// tile are copied by one thread into a ring of F + 3 shared-memory slots with
// tensor copies (cp.async.bulk.tensor, 4-D map over the padded array with its
// rows grouped by x mod 4: 20 positions x 4 residues x rows), two planes ahead
// of the march.  The centre-only data of each updated node (flags, stencil
// class, f or g) are loaded into registers one march step ahead.
//
// A pass reads its fields from one set of arrays and writes its tile to
// another (the FP32 scratch fields RU, RP are free during smoothing):
//   pass 0: (U, P) -> RU;   pass 1: (RU, P) -> (U, RP);   pass 2: (U, RP) -> P,
// so no CTA's write-back can reach a plane another CTA has yet to stage.
//
// Every mbarrier wait is bounded (FusedArgs::polls tests); a CTA whose wait
// runs out writes HHG_TILE_TIMEOUT into the error word, waits (with a bound
// of FUSED_DRAIN_POLLS) for every copy it issued, and returns; if that drain
// also runs out it writes HHG_TILE_DRAIN_TIMEOUT (copies may still land in
// its shared memory: the host treats the mesh as failed).
#include <string>

#include "../../include/hhg_stokes.h"
#include "hhg_kernels.h"
#include "hhg_node_ops.cuh"
#include "hhg_tma.cuh"

namespace hhg {

namespace {

constexpr int FQ = 20;       // staged positions per residue (80 entries per row)
constexpr int FBX = 4 * FQ;  // staged entries per row
constexpr long long FUSED_DRAIN_POLLS = 1ll << 28;

template <int KIND>
__host__ __device__ constexpr int pass_phases() {
  return KIND == 0 ? 4 : 3;
}
__host__ __device__ constexpr int pass_slots(int F) { return F + 3; }

// Colour of phase q of a pass, and its work: 0 velocity, 1 velocity then
// pressure, 2 pressure.
template <int KIND>
__device__ __forceinline__ int phase_colour(int q) {
  return KIND == 0 ? q : (KIND == 1 ? 2 - q : q + 1);
}
template <int KIND>
__device__ __forceinline__ int phase_work(int q) {
  return KIND == 0 ? 0 : (KIND == 1 ? (q == 2 ? 1 : 0) : 2);
}

// Shared-memory view of one field over three consecutive staged planes:
// entry of node (dx, dy, dz) from the centre = pl[dz + 1][e[dx + 1] + FBX dy].
struct RingNb {
  const float* pl[3];
  int e[3];
  __device__ __forceinline__ float operator()(int dx, int dy, int dz) const { return pl[dz + 1][e[dx + 1] + FBX * dy]; }
};

// Centre data of the node a thread updates in one phase.
struct Centre {
  int64_t c;    // padded index (valid when fl != 0)
  float f[3];   // velocity right-hand side
  float g;      // pressure right-hand side
  uint16_t cls; // stencil class (F_IRR nodes)
  uint8_t fl;   // node flags, 0 = nothing to do
};

}  // namespace

template <int KIND>
__global__ void __launch_bounds__(FUSED_MAX_THREADS, 1)
    k_uzawa_pass(const __grid_constant__ TileMaps tm, LevelDev<float> L, FusedArgs a, float inv6nuh, float omc) {
  pdl_enter();
  constexpr int F = pass_phases<KIND>();
  constexpr int NS = pass_slots(F);
  extern __shared__ __align__(128) unsigned char sm[];
  float* fb = reinterpret_cast<float*>(sm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + sizeof(float) * (size_t)NS * 4 * a.fstride);
  const int m = blockIdx.x, b = blockIdx.y;
  const int P0 = 16 * m;                          // first staged position (16-byte aligned in FP32)
  const int x_lo = m == 0 ? 0 : 64 * m + 3;       // the tile's nodes in x
  const int x_hi = min(64 * m + 67, L.nx);
  const int y_lo = b * a.ty, y_hi = min(y_lo + a.ty, L.ny);
  const int jb = y_lo - F;                        // node row of staged row 0
  const int t = threadIdx.x;
  const int r = t / FQ, pb = t - r * FQ;
  const bool live = r < a.by;
  const int j = jb + r;
  const int nz = L.nz;
  const uint32_t slot_bytes = (uint32_t)(4 * FBX * a.by * sizeof(float));

  auto field = [&](int slot, int f) { return fb + (size_t)(slot * 4 + f) * a.fstride; };
  auto issue = [&](int zp) {  // padded plane zp into its slot (thread 0)
    const int s = zp % NS;
    fence_proxy_async_smem();
    // (a.extra_tx: tests announce more bytes than plane 0 delivers, so that
    // the first wait runs out while the real copies land)
    mbar_expect(&bar[s], slot_bytes + (zp == 0 ? (uint32_t)a.extra_tx : 0u));
#pragma unroll
    for (int f = 0; f < 4; ++f) tma_load_4d(field(s, f), &tm.m[f], P0, 0, jb + 1, zp, &bar[s]);
  };

  if (t == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s]);
    mbar_init_fence();
  }
  __syncthreads();
  const int last_zp = nz + 1;  // padded planes 0 .. nz + 1
  int issued = 0, waited = 0;
  if (t == 0)
    for (; issued < 4 && issued <= last_zp; ++issued) issue(issued);
  issued = min(4, last_zp + 1);

  // the node of phase q on march step s, and its centre data.  The loads
  // depend on the node's indices only (never on loaded values), so a march
  // step issues all of the next step's loads back to back and first uses
  // them one step later.
  auto fetch = [&](int s, int q, Centre& cd) {
    cd.fl = 0;
    const int k = s - q;
    if (!live || k < 0 || k >= nz || j < 0 || j >= L.ny) return;
    const int d = F - 1 - q;
    if (j < y_lo - d || j >= y_hi + d) return;
    const int rho = (phase_colour<KIND>(q) - j - k + 1) & 3;
    const int i = 4 * (P0 + pb) + rho - 1;
    if (i < 0 || i >= L.nx || i < x_lo - d || i >= x_hi + d) return;
    const int64_t c = pad_index(L.px, L.pxy, i, j, k);
    const int w = phase_work<KIND>(q);
    cd.c = c;
    cd.fl = __ldg(L.flags + c);
    if (w != 2) {
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) cd.f[dd] = __ldg(L.f[dd] + c);
    }
    if (w != 0) cd.g = __ldg(L.g + c);
    cd.cls = __ldg(L.cls + c);
  };

  Centre cur[F], nxt[F];
#pragma unroll
  for (int q = 0; q < F; ++q) fetch(0, q, cur[q]);

  const int steps = nz + F - 1;
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int q = 0; q < F; ++q) fetch(s + 1, q, nxt[q]);
    // planes up to padded s + 2 must have landed (waited: the first plane this
    // thread has not seen complete)
    bool ok = true;
    while (ok && waited <= s + 2 && waited <= last_zp) {
      ok = mbar_wait(&bar[waited % NS], (uint32_t)((waited / NS) & 1), a.polls);
      if (ok) ++waited;
    }
    if (!__syncthreads_and(ok)) {
      if (t == 0) {
        // a copy did not land in time: report it, and let every copy still in
        // flight land before the CTA's shared memory is released
        atomicExch(a.err, (unsigned)HHG_TILE_TIMEOUT);
        if (a.extra_tx && waited == 0) mbar_complete_tx(&bar[0], (uint32_t)a.extra_tx);
        bool drained = true;
        for (int w = waited; w < issued && drained; ++w)
          drained = mbar_wait(&bar[w % NS], (uint32_t)((w / NS) & 1), FUSED_DRAIN_POLLS);
        if (!drained) atomicExch(a.err, (unsigned)HHG_TILE_DRAIN_TIMEOUT);
      }
      __syncthreads();
      return;
    }
#pragma unroll
    for (int q = 0; q < F; ++q) {
      const Centre& cd = cur[q];
      const int work = phase_work<KIND>(q);
      if (cd.fl & (work == 2 ? F_ACT : (work == 1 ? (F_ACT | F_VFREE) : F_VFREE))) {
        const int k = s - q;
        const int rho = (phase_colour<KIND>(q) - j - k + 1) & 3;
        float* pl[3][4];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int f = 0; f < 4; ++f) pl[dz][f] = field((k + dz) % NS, f);
        const int ec = r * FBX + rho * FQ + pb;
        const int e[3] = {rho == 0 ? ec + 3 * FQ - 1 : ec - FQ, ec, rho == 3 ? ec - 3 * FQ + 1 : ec + FQ};
        const RingNb u[3] = {RingNb{{pl[0][0], pl[1][0], pl[2][0]}, {e[0], e[1], e[2]}},
                             RingNb{{pl[0][1], pl[1][1], pl[2][1]}, {e[0], e[1], e[2]}},
                             RingNb{{pl[0][2], pl[1][2], pl[2][2]}, {e[0], e[1], e[2]}}};
        const RingNb p{{pl[0][3], pl[1][3], pl[2][3]}, {e[0], e[1], e[2]}};
        const float* w = (cd.fl & F_IRR) ? L.wt + (int64_t)W_STRIDE * cd.cls : nullptr;
        if (work != 2 && (cd.fl & F_VFREE)) {
          float nu[3];
          if (!(cd.fl & F_IRR))
            vel_regular_value(L, cd.f, u, p, inv6nuh, nu);
          else
            vel_irr_value(L, w, cd.f, u, p, nu);
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) pl[1][dd][ec] = nu[dd];
        }
        if (work != 0 && (cd.fl & F_ACT)) {
          const float pc = pl[1][3][ec];
          pl[1][3][ec] = (cd.fl & F_IRR) ? pres_irr_value(L, w, cd.g, u, p, pc)
                                         : pres_regular_value(L, cd.g, u, p, pc, omc);
        }
      }
      __syncthreads();
    }
    // plane s - F + 1 is final: write the tile's nodes to the output fields
    const int kw = s - F + 1;
    if (kw >= 0 && live && j >= y_lo && j < y_hi) {
      const int sl = (kw + 1) % NS;
#pragma unroll
      for (int rho = 0; rho < 4; ++rho) {
        const int i = 4 * (P0 + pb) + rho - 1;
        if (i < x_lo || i >= x_hi) continue;
        const int64_t c = pad_index(L.px, L.pxy, i, j, kw);
        const int ec = r * FBX + rho * FQ + pb;
        if (KIND != 2) {
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) a.out_u[dd][c] = field(sl, dd)[ec];
        }
        if (KIND != 0) a.out_p[c] = field(sl, 3)[ec];
      }
    }
    __syncthreads();
    // the slot of padded plane s - F + 1 is free: stage padded plane s + 4 into it
    if (t == 0 && s + 4 <= last_zp) issue(s + 4);
    if (s + 4 <= last_zp) issued = s + 5;
#pragma unroll
    for (int q = 0; q < F; ++q) cur[q] = nxt[q];
  }
}

// ---- host side ------------------------------------------------------------------------------

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_maps(const LevelDev<float>& L, const float* const* f, int by, TileMaps& out, std::string& err) {
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
  // 4-D over the padded array: (px / 4 positions, 4 residues, py rows, pz planes)
  const cuuint64_t dims[4] = {(cuuint64_t)(L.px / 4), 4, (cuuint64_t)(L.pxy / L.px), (cuuint64_t)(L.nalloc / L.pxy)};
  const cuuint64_t strides[3] = {(cuuint64_t)(L.px / 4) * sizeof(float), (cuuint64_t)L.px * sizeof(float),
                                 (cuuint64_t)L.pxy * sizeof(float)};
  const cuuint32_t box[4] = {FQ, 4, (cuuint32_t)by, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int q = 0; q < 4; ++q) {
    if (((uintptr_t)f[q] & 15) || (strides[0] & 15) || (strides[1] & 15) || (strides[2] & 15)) {
      err = "field not aligned for tensor copies";
      return HHG_EINVAL;
    }
    const CUresult r = encode(&out.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)f[q], dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      return HHG_ECUDA;
    }
  }
  return HHG_OK;
}

int pass_threads(int by) { return ((by * FQ + 31) / 32) * 32; }
size_t pass_fstride(int by) { return (size_t)((by * FBX + 31) / 32) * 32; }  // floats, 128-byte multiple
size_t pass_smem(int F, int by) {
  return sizeof(float) * (size_t)pass_slots(F) * 4 * pass_fstride(by) + sizeof(uint64_t) * pass_slots(F);
}

int g_sms = 0;
size_t g_smem_optin = 0;

}  // namespace

int fused_tiles_x(int nx) { return nx <= 67 ? 1 : (nx - 67 + 63) / 64 + 1; }

// Rows per tile of each pass: the efficiency (tile rows / staged rows) x
// (CTAs / the slots of the waves they need) is maximised over the row counts
// whose ring fits the shared memory.
int plan_fused(const LevelDev<float>& L, int ty_override, FusedPlan& P, std::string& err) {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g_smem_optin = (size_t)optin;
    if (g_sms <= 0 || optin <= 0) {
      err = "device attributes unavailable";
      return HHG_ECUDA;
    }
  }
  P.ntx = fused_tiles_x(L.nx);
  for (int kind = 0; kind < 3; ++kind) {
    const int F = kind == 0 ? 4 : 3;
    double best = -1.0;
    int best_ty = 0;
    for (int ty = 1; ty + 2 * F <= 32; ++ty) {
      const int by = ty + 2 * F;
      const size_t sm = pass_smem(F, by);
      if (sm > g_smem_optin || pass_threads(by) > FUSED_MAX_THREADS) break;
      if (ty_override > 0 && ty != ty_override) continue;
      int res = (int)((g_smem_optin + 1024) / (sm + 1024));
      res = std::min(res, 2048 / pass_threads(by));
      res = std::max(res, 1);
      const int64_t ctas = (int64_t)P.ntx * ((L.ny + ty - 1) / ty);
      const int64_t slots = (int64_t)g_sms * res;
      const int64_t waves = (ctas + slots - 1) / slots;
      const double eff = (double)ty / by * (double)ctas / (double)(waves * slots);
      if (eff > best) {
        best = eff;
        best_ty = ty;
      }
    }
    if (!best_ty) {
      err = "no tile height fits the fused passes";
      return HHG_EINVAL;
    }
    P.ty[kind] = best_ty;
    P.by[kind] = best_ty + 2 * F;
    P.nty[kind] = (L.ny + best_ty - 1) / best_ty;
  }
  const float* in[3][4] = {{L.u[0], L.u[1], L.u[2], L.p}, {L.r[0], L.r[1], L.r[2], L.p}, {L.u[0], L.u[1], L.u[2], L.rp}};
  for (int kind = 0; kind < 3; ++kind) {
    int rc = encode_maps(L, in[kind], P.by[kind], P.maps[kind], err);
    if (rc) return rc;
  }
  return HHG_OK;
}

template <int KIND>
static void launch_pass(const FusedPlan& P, const LevelDev<float>& L, unsigned* err, long long polls, int extra_tx,
                        cudaStream_t s) {
  constexpr int F = pass_phases<KIND>();
  FusedArgs a{};
  a.by = P.by[KIND];
  a.ty = P.ty[KIND];
  a.fstride = (int)pass_fstride(a.by);
  a.polls = polls;
  a.extra_tx = extra_tx;
  a.err = err;
  for (int d = 0; d < 3; ++d) a.out_u[d] = KIND == 0 ? L.r[d] : L.u[d];
  a.out_p = KIND == 1 ? L.rp : L.p;
  const float inv = (float)(1.0 / (6.0 * (double)L.nuh));
  const float omc = (float)((double)L.omega / (6.0 * (double)L.c));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P.ntx, (unsigned)P.nty[KIND], 1);
  cfg.blockDim = dim3((unsigned)pass_threads(a.by));
  cfg.dynamicSmemBytes = pass_smem(F, a.by);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_uzawa_pass<KIND>, P.maps[KIND], L, a, inv, omc);
}

void launch_uzawa_pass(const FusedPlan& P, const LevelDev<float>& L, int kind, unsigned* err, long long polls,
                       int extra_tx, cudaStream_t s) {
  if (kind == 0)
    launch_pass<0>(P, L, err, polls, extra_tx, s);
  else if (kind == 1)
    launch_pass<1>(P, L, err, polls, extra_tx, s);
  else
    launch_pass<2>(P, L, err, polls, extra_tx, s);
}

void prepare_fused() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncSetAttribute(k_uzawa_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaFuncSetAttribute(k_uzawa_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaFuncSetAttribute(k_uzawa_pass<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

}  // namespace hhg
