// C ABI of the solver (include/hhg_stokes.h): hierarchy set-up, the V_var
// cycle driver (Sec. 3.3-3.6), FP64 and FP32-in-FP64-refinement solves, the
// adjoint gradient, and step-level hooks for parity tests.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/hhg_stokes.h"
#include "hhg_kernels.h"
#include "hhg_lattice.h"

using namespace hhg;

namespace {

thread_local std::string g_create_error;

struct LevelHost {
  int level = 0;
  LevelShape sh{};
  int64_t px = 0, py = 0, pz = 0, nalloc = 0;
  double h = 0, hT2 = 0;
  std::vector<uint8_t> flags;  // lattice order
  uint8_t* d_flags = nullptr;
  uint16_t* d_cls = nullptr;   // padded stencil class of boundary nodes
  double* d_wt64 = nullptr;    // class row tables
  float* d_wt32 = nullptr;
  double* d_wt2_64 = nullptr;  // D form: velocity-block row tables (W2_STRIDE per class)
  float* d_wt2_32 = nullptr;
  int n_classes = 0;
  int64_t n_vel = 0, n_pres = 0;
  bool fused = false;  // FP32 Uzawa steps as the three colour-fused passes (hhg_fused.cu)
  FusedPlan fz{};
  int64_t ndir = 0;                  // Dirichlet nodes of the level: lattice and padded indices, values
  int64_t* d_dir_lat = nullptr;
  int64_t* d_dir_pad = nullptr;
  double* d_dir_val = nullptr;
  int64_t nirr = 0;                  // F_IRR nodes of the level, (k << 42) | (j << 21) | i
  int64_t* d_irr = nullptr;
  int32_t* d_list = nullptr;         // node lists of the cluster-resident cycle (ResidentCycle::lists)
  int32_t loff[RES_LISTS + 1] = {};  // their offsets
  double* mem64 = nullptr;
  float* mem32 = nullptr;
  LevelDev<double> d64{};
  LevelDev<float> d32{};
};

template <class T>
void bind_fields(LevelDev<T>& L, T* base, int64_t nalloc) {
  for (int d = 0; d < 3; ++d) {
    L.u[d] = base + (int64_t)d * nalloc;
    L.f[d] = base + (int64_t)(4 + d) * nalloc;
    L.r[d] = base + (int64_t)(8 + d) * nalloc;
  }
  L.p = base + 3 * nalloc;
  L.g = base + 7 * nalloc;
  L.rp = base + 11 * nalloc;
}

}  // namespace

struct hhg_mesh {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hhg_options opt{};
  MacroLattice macro;
  int finest = 0, coarsest = 0;
  int small_top[2] = {-1, -1};  // top level of the fused coarse-levels cycle, FP64 / FP32 (-1: none)
  int res_top[2] = {-1, -1};    // top level of the cluster-resident cycle, FP64 / FP32 (-1: none)
  unsigned res_nb[2] = {16, 16};  // its cluster size
  size_t res_smem[2] = {0, 0};    // its shared-memory limit per CTA
  unsigned small_cluster[2] = {1, 8};  // CTAs of the fused team, FP64 / FP32
  std::vector<LevelHost> lv;
  uint8_t* d_mmask = nullptr;
  int64_t ndir = 0;               // the finest level's Dirichlet list (aliases of lv[finest]'s)
  int64_t* d_dir_lat = nullptr;
  int64_t* d_dir_pad = nullptr;
  double* d_dir_val = nullptr;
  double* d_stage = nullptr;  // 3 n doubles (finest)
  double* d_partial = nullptr;
  double* d_ir_partial = nullptr;  // per-block partial norms of the fixed-point residual (finest level)
  double* d_scalars = nullptr;  // [0] norm2, [1..2] moments, [3..4] g-mean, [5..7] coarse info
  double* h_scalars = nullptr;  // pinned mirror
  unsigned long long* d_fxmax = nullptr;  // fixed-point state: FxState's mx, maxq and exp (12 words)
  FxIterate fx{};                          // fixed-point finest iterate (FP32+IR mode)
  int64_t* d_fx = nullptr;
  int64_t* d_fx_irr = nullptr;  // F_IRR nodes of the finest level (FxState::irr; alias of lv[finest].d_irr)
  int64_t n_fx_irr = 0;
  unsigned long long* d_rhs_fx = nullptr;  // right-hand side quantization: maxima [0..8), shifts
  double* d_coarse = nullptr;  // coarse-solve scratch
  CoarseSys coarse_sys{};       // compact coarsest-level system (device arrays)
  void* d_coarse_sys = nullptr;  // one allocation holding its arrays
  double* d_backup = nullptr;  // 8 finest FP64 fields (adjoint)
  // cycle graphs: FP64, FP32+IR, FP32+IR with the FP64 update (first cycle
  // from an iterate with an all-zero field)
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  int64_t graph_launches[3] = {0, 0, 0};
  unsigned long long h_fxmax[4] = {0, 0, 0, 0};  // max |x| per field of the last quantization
  bool rhs_set = false;
  bool broken = false;  // a fused pass could not drain its copies (tile_status)
  int64_t launches = 0;
  int64_t fx_recoveries = 0;  // fixed-point cycles redone in FP64 (fx_recover_if_flagged)
  int vroot = -1;             // root level of the V-cycles being enqueued (-1: the finest)
  int vnu = -1;               // their smoothing steps on the root level (-1: nu_pre / nu_post)
  int64_t device_bytes = 0;
  int64_t allocations = 0;  // cudaMalloc / cudaMallocHost calls made for this mesh, temporaries included
  std::string err;
};

namespace {

int fail(hhg_mesh* M, int code, const std::string& msg) {
  if (M) M->err = msg;
  return code;
}

int cuda_fail(hhg_mesh* M, cudaError_t e, const char* where) {
  return fail(M, HHG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(M, e_, #call); \
  } while (0)

int dalloc(hhg_mesh* M, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(M, HHG_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
  }
  M->device_bytes += (int64_t)bytes;
  M->allocations += 1;
  return HHG_OK;
}

void fill_coefs(hhg_mesh* M, LevelHost& H) {
  auto set = [&](auto& L) {
    using T = std::remove_reference_t<decltype(L.nuh)>;
    L.nx = H.sh.nx;
    L.ny = H.sh.ny;
    L.nz = H.sh.nz;
    L.level = H.level;
    L.mx = M->macro.mx;
    L.my = M->macro.my;
    L.mz = M->macro.mz;
    L.px = H.px;
    L.pxy = H.px * H.py;
    L.nalloc = H.nalloc;
    L.flags = H.d_flags;
    L.mmask = M->d_mmask;
    L.cls = H.d_cls;
    L.nuh = (T)(M->opt.nu * H.h);
    L.c = (T)(M->opt.delta * H.hT2 * H.h);
    L.h2 = (T)(H.h * H.h);
    L.h3 = (T)(H.h * H.h * H.h);
    L.dh2 = (T)(M->opt.delta * H.hT2);
    L.omega = (T)M->opt.omega;
    const int64_t lim = M->opt.spec_max_nodes != 0 ? M->opt.spec_max_nodes : SPEC_MAX_NODES;
    L.spec = lim > 0 && H.sh.n() < lim;
    const int want = M->opt.colour_block_z;
    // one plane per block: measured 4-5 % faster per FP32 Uzawa step than two on the level-8 and level-9 cubes
    L.cbz = want == 1 || want == 2 || want == 4 ? want : 1;
    L.nq = (int)((H.sh.nx + 3) / 4);
    L.nq_mul = L.nq == 1 ? 0 : ~0ull / (uint64_t)L.nq + 1;
    // two nodes per thread in the FP32 colour kernels of the flags-first (large)
    // levels: an option, off by default (measured on GB300, level-9 FP32 Uzawa
    // step 9.30 ms with pairs against 6.70 ms without: the colour kernels are
    // bound by the loads in flight, and the pair kernels' 64 registers and the
    // unaligned x-neighbour pairs of two residues in four cost more than the
    // halved load count saves)
    L.pairs = sizeof(T) == 4 && M->opt.colour_pairs > 0 && !L.spec;
    {
      const int32_t q = M->opt.quad_min_nodes;
      // four nodes per thread pays on the largest levels only (measured: level 9
      // 5.10 -> 4.30 ms, level 8 unchanged, level 7 0.100 -> 0.114 ms)
      const int64_t lim = q == 0 ? ((int64_t)1 << 25) : (q < 0 ? std::numeric_limits<int64_t>::max() : (int64_t)q);
      L.quad = sizeof(T) == 4 && H.sh.n() >= lim ? 1 : 0;  // FP64: 176 registers, no gain
    }
    L.nq2 = L.nq / 2 + 1;
    L.nq2_mul = L.nq2 == 1 ? 0 : ~0ull / (uint64_t)L.nq2 + 1;
  };
  set(H.d64);
  set(H.d32);
  H.d64.wt = H.d_wt64;
  H.d32.wt = H.d_wt32;
  H.d64.wt2 = H.d_wt2_64;
  H.d32.wt2 = H.d_wt2_32;
}

int ensure32(hhg_mesh* M) {
  for (int l = M->coarsest; l <= M->finest; ++l) {
    LevelHost& H = M->lv[l];
    if (H.mem32) continue;
    int rc = dalloc(M, (void**)&H.mem32, sizeof(float) * 12 * (size_t)H.nalloc);
    if (rc) return rc;
    CK(cudaMemsetAsync(H.mem32, 0, sizeof(float) * 12 * (size_t)H.nalloc, M->stream));
    bind_fields(H.d32, H.mem32, H.nalloc);
    const int64_t lim = M->opt.fused_min_nodes != 0 ? M->opt.fused_min_nodes : FUSED_MIN_NODES;
    H.fused = lim > 0 && H.sh.n() >= lim;
    if (H.fused && (rc = plan_fused(H.d32, M->opt.fused_tile_rows, H.fz, M->err))) return rc;
  }
  if (M->opt.ir_fixed_point && !M->d_fx) {
    const LevelHost& H = M->lv[M->finest];
    int rc = dalloc(M, (void**)&M->d_fx, sizeof(int64_t) * 4 * (size_t)H.nalloc);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d) M->fx.u[d] = M->d_fx + (int64_t)d * H.nalloc;
    M->fx.p = M->d_fx + 3 * H.nalloc;
    if ((rc = dalloc(M, (void**)&M->d_fxmax, 12 * sizeof(unsigned long long)))) return rc;
    CK(cudaMemsetAsync(M->d_fxmax, 0, 12 * sizeof(unsigned long long), M->stream));
  }
  return HHG_OK;
}

// Fixed-point state: maxima and shifts in d_fxmax, the flag word in the
// scalar block (read back with the norm after every cycle).
FxState fx_state(hhg_mesh* M) {
  return FxState{M->d_fxmax, M->d_fxmax + 4, reinterpret_cast<int*>(M->d_fxmax + 8),
                 reinterpret_cast<unsigned*>(M->d_scalars + 14), M->d_fx_irr, M->n_fx_irr};
}

// ---- enqueue helpers (no synchronisation; graph-capturable) -------------------

template <class T>
LevelDev<T>& view(hhg_mesh* M, int l);
template <>
LevelDev<double>& view<double>(hhg_mesh* M, int l) { return M->lv[l].d64; }
template <>
LevelDev<float>& view<float>(hhg_mesh* M, int l) { return M->lv[l].d32; }

// Error word of the fused passes (the last slot of the scalar block).
unsigned* err_word(hhg_mesh* M) { return reinterpret_cast<unsigned*>(M->d_scalars + 15); }

template <class T>
void enq_vel_sweep(hhg_mesh* M, int l, bool forward) {
  for (int q = 0; q < 4; ++q) launch_vel_colour<T>(view<T>(M, l), forward ? q : 3 - q, M->stream);
  M->launches += 4;
}

template <class T>
void enq_pres_sweep(hhg_mesh* M, int l) {
  for (int q = 0; q < 4; ++q) launch_pres_colour<T>(view<T>(M, l), q, M->stream);
  M->launches += 4;
}

// The colour kernels of an Uzawa step on their own: the forward velocity
// sweep with f - B^T p formed at each node, and the pressure sweep with
// B u - g formed at each node.
template <class T>
void enq_vel_sweep_f(hhg_mesh* M, int l) {
  const LevelDev<T>& L = view<T>(M, l);
  for (int q = 0; q < 4; ++q) launch_vel_colour_rhs<T>(L, q, M->stream);
  M->launches += 4;
}

template <class T>
void enq_pres_sweep_f(hhg_mesh* M, int l) {
  const LevelDev<T>& L = view<T>(M, l);
  for (int q = 0; q < 4; ++q) launch_pres_colour_rhs<T>(L, q, M->stream);
  M->launches += 4;
}

// One inexact Uzawa step (Sec. 3.3): velocity SHGS on f - B^T p (colours
// 0,1,2,3 then 3,2,1,0), then the relaxed pressure sweep on B u - g.  The
// backward colour 3 repeats the forward one with unchanged neighbours and a
// node's new value does not depend on its old one, so it is skipped (the
// result is identical).  FP32 forms f - B^T p at each node inside the colour
// kernels; FP64, bound by its arithmetic rate, stores it once per step.  The
// pressure colours form B u - g at each node (every node is updated once).
// The last velocity colour and the first pressure colour share a launch
// (k_vel_pres_colour0): 10 launches per step.
// The three colour-fused passes of an FP32 Uzawa step (hhg_fused.cu); kind
// -1 runs all three.
void enq_uzawa_fused(hhg_mesh* M, int l, int kind = -1) {
  const long long polls = M->opt.wait_poll_limit > 0 ? M->opt.wait_poll_limit : FUSED_WAIT_POLLS;
  for (int k = 0; k < 3; ++k)
    if (kind < 0 || kind == k) {
      launch_uzawa_pass(M->lv[l].fz, view<float>(M, l), k, err_word(M), polls, M->opt.fused_wait_test ? 16 : 0,
                        M->stream);
      M->launches += 1;
    }
}

template <class T>
void enq_uzawa(hhg_mesh* M, int l) {
  const LevelDev<T>& L = view<T>(M, l);
  const bool ru = sizeof(T) != 4;
  if (!ru && M->lv[l].fused) {
    enq_uzawa_fused(M, l);
    return;
  }
  if (ru) {
    launch_vel_rhs<T>(L, M->stream);
    M->launches += 1;
  }
  // velocity colours 0 1 2 3 2 1, then backward colour 0 with pressure colour 0, then pressure 1 2 3
  for (int q = 0; q < 6; ++q) {
    const int colour = q < 4 ? q : 6 - q;
    ru ? launch_vel_colour<T>(L, colour, M->stream) : launch_vel_colour_rhs<T>(L, colour, M->stream);
  }
  launch_vel_pres_colour0<T>(L, ru, M->stream);
  for (int q = 1; q < 4; ++q) launch_pres_colour_rhs<T>(L, q, M->stream);
  M->launches += 10;
}

template <class T>
void enq_coarse(hhg_mesh* M) {
  CoarseParams prm{M->opt.coarse_minres_max, M->opt.coarse_minres_rtol, M->opt.coarse_cg_max, M->opt.coarse_cg_rtol};
  launch_coarse_solve<T>(M->coarse_sys, view<T>(M, M->coarsest), M->d_coarse, prm, M->d_scalars + 5, M->stream);
  M->launches += 1;
}

// Smoothing steps on level l of a V_var cycle rooted at M->vroot (Sec. 3.5;
// Sec. 5 for the cycles of FMG, rooted below the finest level).
template <class T>
int nu_steps(hhg_mesh* M, int l, bool pre) {
  const int base = M->vnu >= 0 ? M->vnu : (pre ? M->opt.nu_pre : M->opt.nu_post);
  const int root = M->vroot >= 0 ? M->vroot : M->finest;
  return base + M->opt.var_increment * (root - l);
}

template <class T>
int nu_steps(hhg_mesh* M, int l, bool pre);

template <class T>
void enq_small_cycle(hhg_mesh* M) {
  SmallCycle<T> S;
  std::memset(&S, 0, sizeof(S));
  S.nblocks = M->small_cluster[sizeof(T) == 4];
  S.nlev = M->small_top[sizeof(T) == 4] - M->coarsest + 1;
  for (int q = 0; q < S.nlev; ++q) {
    const int l = M->coarsest + q;
    S.lv[q] = view<T>(M, l);
    S.nu_pre[q] = nu_steps<T>(M, l, true);
    S.nu_post[q] = nu_steps<T>(M, l, false);
    S.inv6nuh[q] = (T)(1.0 / (6.0 * (double)S.lv[q].nuh));
    S.omc[q] = (T)((double)S.lv[q].omega / (6.0 * (double)S.lv[q].c));
  }
  S.cs = M->coarse_sys;
  S.scratch = M->d_coarse;
  S.prm = CoarseParams{M->opt.coarse_minres_max, M->opt.coarse_minres_rtol, M->opt.coarse_cg_max,
                       M->opt.coarse_cg_rtol};
  S.info = M->d_scalars + 5;
  launch_small_cycle<T>(S, M->stream);
  M->launches += 1;
}

// Node lists of a level for the cluster-resident cycle: list 8 kind + 2 colour
// + boundary holds the velocity (kind 0, F_VFREE) or pressure (kind 1, F_ACT)
// nodes of colour (i + j + k) mod 4, regular (boundary 0) or F_IRR
// (boundary 1), as (k << 20) | (j << 10) | i in lattice order.  The fused
// colour-0 phase walks the pressure lists, so the lists are built only where
// every velocity node is active and every regular active node carries a
// velocity (a Dirichlet or outflow node lies on the domain boundary, F_IRR).
int build_node_lists(hhg_mesh* M, LevelHost& H) {
  const LevelShape& sh = H.sh;
  if (sh.nx >= 1024 || sh.ny >= 1024 || sh.nz >= 2048) return HHG_OK;
  std::vector<std::vector<int32_t>> lists(RES_LISTS);
  for (int k = 0; k < sh.nz; ++k)
    for (int j = 0; j < sh.ny; ++j)
      for (int i = 0; i < sh.nx; ++i) {
        const uint8_t f = H.flags[i + (int64_t)sh.nx * (j + (int64_t)sh.ny * k)];
        if ((f & F_VFREE) && !(f & F_ACT)) return HHG_OK;
        if ((f & F_ACT) && !(f & F_IRR) && !(f & F_VFREE)) return HHG_OK;
        const int32_t e = (k << 20) | (j << 10) | i;
        const int b = 2 * ((i + j + k) & 3) + ((f & F_IRR) ? 1 : 0);
        if (f & F_VFREE) lists[b].push_back(e);
        if (f & F_ACT) lists[8 + b].push_back(e);
      }
  std::vector<int32_t> all;
  for (int l = 0; l < RES_LISTS; ++l) {
    H.loff[l] = (int32_t)all.size();
    all.insert(all.end(), lists[l].begin(), lists[l].end());
  }
  H.loff[RES_LISTS] = (int32_t)all.size();
  int rc = dalloc(M, (void**)&H.d_list, sizeof(int32_t) * std::max<size_t>(all.size(), 1));
  if (rc) return rc;
  CK(cudaMemcpy(H.d_list, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice));
  return HHG_OK;
}

template <class T>
void fill_resident(hhg_mesh* M, ResidentCycle<T>& S, int top) {
  std::memset(&S, 0, sizeof(S));
  const int pr = sizeof(T) == 4;
  S.nblocks = M->res_nb[pr];
  S.nres = top - M->coarsest;
  for (int q = 0; q <= S.nres; ++q) {
    const int l = M->coarsest + q;
    S.lv[q] = view<T>(M, l);
    S.ncls[q] = M->lv[l].n_classes;
    S.nu_pre[q] = nu_steps<T>(M, l, true);
    S.nu_post[q] = nu_steps<T>(M, l, false);
    S.inv6nuh[q] = (T)(1.0 / (6.0 * (double)S.lv[q].nuh));
    S.omc[q] = (T)((double)S.lv[q].omega / (6.0 * (double)S.lv[q].c));
  }
  for (int q = 1; q <= S.nres; ++q) {
    const LevelHost& H = M->lv[M->coarsest + q];
    S.lists[q] = H.d_list;
    std::memcpy(S.loff[q], H.loff, sizeof(H.loff));
  }
  S.cs = M->coarse_sys;
  S.scratch = M->d_coarse;
  S.prm = CoarseParams{M->opt.coarse_minres_max, M->opt.coarse_minres_rtol, M->opt.coarse_cg_max,
                       M->opt.coarse_cg_rtol};
  S.info = M->d_scalars + 5;
}

template <class T>
void enq_resident_cycle(hhg_mesh* M) {
  ResidentCycle<T> S;
  fill_resident<T>(M, S, M->res_top[sizeof(T) == 4]);
  plan_resident<T>(S, M->res_smem[sizeof(T) == 4], M->res_nb[sizeof(T) == 4]);
  launch_resident_cycle<T>(S, M->stream);
  M->launches += 1;
}

// One V_var cycle rooted at level l (Sec. 3.5).
template <class T>
void enq_vcycle(hhg_mesh* M, int l) {
  if (l == M->coarsest) {
    enq_coarse<T>(M);
    return;
  }
  if (l == M->res_top[sizeof(T) == 4]) {
    enq_resident_cycle<T>(M);
    return;
  }
  if (l == M->small_top[sizeof(T) == 4]) {
    enq_small_cycle<T>(M);
    return;
  }
  for (int s = 0; s < nu_steps<T>(M, l, true); ++s) enq_uzawa<T>(M, l);
  launch_residual<T>(view<T>(M, l), M->stream);
  launch_restrict<T>(view<T>(M, l), view<T>(M, l - 1), M->stream);
  M->launches += 2;
  enq_vcycle<T>(M, l - 1);
  launch_prolong_add<T>(view<T>(M, l), view<T>(M, l - 1), M->stream);
  M->launches += 1;
  for (int s = 0; s < nu_steps<T>(M, l, false); ++s) enq_uzawa<T>(M, l);
}

template <class T>
void enq_project(hhg_mesh* M, int l) {
  launch_mass_moments<T>(view<T>(M, l), M->d_partial, M->d_scalars + 1, M->stream);
  launch_project<T>(view<T>(M, l), M->d_scalars + 1, M->stream);
  M->launches += 3;
}

// FP64 cycle body: V-cycle, mean projection, residual and its norm.
void enq_cycle64(hhg_mesh* M) {
  enq_vcycle<double>(M, M->finest);
  if (!M->macro.has_outflow) enq_project<double>(M, M->finest);
  launch_residual<double>(M->lv[M->finest].d64, M->stream);
  launch_residual_norm2<double>(M->lv[M->finest].d64, M->d_partial, M->d_scalars, M->stream);
  M->launches += 3;
}

// FP64 residual of the finest iterate into the FP32 right-hand side, its
// squared norm into d_scalars[0]; in fixed point, from_update: of the
// iterate k_fx_update left (checked), else of the FP64 iterate (quantized).
void enq_ir_residual(hhg_mesh* M, bool from_update) {
  LevelHost& H = M->lv[M->finest];
  if (M->opt.ir_fixed_point) {
    launch_ir_residual_fx(H.d64, M->fx, H.d32, fx_state(M), from_update, M->d_ir_partial, M->d_scalars, M->stream);
    M->launches += from_update ? 4 : 6;
  } else {
    launch_ir_residual(H.d64, H.d32, M->d_partial, M->d_scalars, M->stream);
    M->launches += 2;
  }
}

// Free slip (Sec. 6.1): after a refinement update the slip velocities of the
// iterate are made tangential again in FP64 (the FP32 correction is
// tangential only to FP32 rounding); fixed_point: on the finest level's
// fixed-point iterate.
void enq_slip_fix(hhg_mesh* M, int level, bool fixed_point) {
  if (!M->macro.has_slip) return;
  LevelHost& H = M->lv[level];
  if (fixed_point)
    launch_slip_fix_fx(M->fx, H.d64, fx_state(M), M->stream);
  else
    launch_slip_fix(H.d64, H.d_irr, H.nirr, M->stream);
  M->launches += 1;
}

// FP32+IR cycle body: correction V-cycle in FP32 from zero on the FP32
// residual, x += e (in fixed point: Q += round(e 2^s)), FP64 residual ->
// FP32 right-hand side.  On a
// mesh without outflow the residual does not change under constant shifts
// of the pressure (B^T 1 = 0, C 1 = 0), so the mean projection is applied
// once, to the final iterate (do_solve).
void enq_cycle32(hhg_mesh* M, bool fp64_update = false) {
  LevelHost& H = M->lv[M->finest];
  launch_zero<float>(H.d32, 0, M->stream);
  enq_vcycle<float>(M, M->finest);
  if (M->opt.ir_fixed_point && !fp64_update) {
    launch_fx_update(M->fx, H.d32, fx_state(M), H.nalloc, M->stream);
    M->launches += 1;
    enq_slip_fix(M, M->finest, true);
    enq_ir_residual(M, true);
  } else {
    // FP64 update; in fixed point the iterate is then quantized afresh
    launch_ir_update(H.d64, H.d32, M->stream);
    M->launches += 1;
    enq_slip_fix(M, M->finest, false);
    enq_ir_residual(M, false);
  }
}

// Reads the error word copied with the scalar block: a fused pass whose
// tensor copy did not complete in time leaves HHG_TILE_TIMEOUT there (the
// word is cleared for the next call; the level's fields are then
// undefined), HHG_TILE_DRAIN_TIMEOUT if the CTA could not even wait for its
// copies to land (the mesh is marked failed: every later call returns
// HHG_ECUDA).
int tile_status(hhg_mesh* M) {
  if (M->broken) return fail(M, HHG_ECUDA, "a fused pass could not drain its tensor copies; destroy the mesh");
  const unsigned w = *reinterpret_cast<const unsigned*>(M->h_scalars + 15);
  if (!w) return HHG_OK;
  CK(cudaMemsetAsync(err_word(M), 0, sizeof(unsigned), M->stream));
  CK(cudaStreamSynchronize(M->stream));
  *reinterpret_cast<unsigned*>(M->h_scalars + 15) = 0;
  if (w == HHG_TILE_DRAIN_TIMEOUT) {
    M->broken = true;
    return fail(M, HHG_ECUDA, "a fused pass could not drain its tensor copies; destroy the mesh");
  }
  return fail(M, HHG_ECUDA, "a fused colour pass gave up waiting for its tensor copies");
}

// After a fixed-point cycle whose update or residual check raised a flag
// (h_scalars just read back): the FP64 iterate is rebuilt as the iterate
// before the update plus the correction in FP64, requantized with fresh
// shifts, and its residual and norm recomputed (h_scalars refreshed).
int fx_recover_if_flagged(hhg_mesh* M) {
  const unsigned w = *reinterpret_cast<const unsigned*>(M->h_scalars + 14);
  if (!w) return HHG_OK;
  LevelHost& H = M->lv[M->finest];
  const FxState st = fx_state(M);
  launch_fx_to_fp64(H.d64, M->fx, H.d32, st, true, M->stream);
  enq_slip_fix(M, M->finest, false);
  enq_ir_residual(M, false);  // clears the flag
  M->launches += 1;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  M->fx_recoveries += 1;
  return HHG_OK;
}

// The FP64 iterate from the fixed-point one (end of an FP32+IR solve).
void fx_materialize(hhg_mesh* M) {
  LevelHost& H = M->lv[M->finest];
  launch_fx_to_fp64(H.d64, M->fx, H.d32, fx_state(M), false, M->stream);
  M->launches += 1;
}

// One solver cycle; fp64_update: an FP32+IR cycle whose update is done in
// FP64 (the fixed-point iterate then requantized).
int run_cycle(hhg_mesh* M, int mode, double* norm2, bool fp64_update = false) {
  const int gi = mode == 0 ? 0 : (fp64_update && M->opt.ir_fixed_point ? 2 : 1);
  if (M->opt.use_graphs) {
    if (!M->graph[gi]) {
      cudaGraph_t g;
      const int64_t before = M->launches;
      CK(cudaStreamBeginCapture(M->stream, cudaStreamCaptureModeThreadLocal));
      if (mode == 0)
        enq_cycle64(M);
      else
        enq_cycle32(M, gi == 2);
      cudaError_t e = cudaStreamEndCapture(M->stream, &g);
      if (e != cudaSuccess) return cuda_fail(M, e, "graph capture");
      M->graph_launches[gi] = M->launches - before;
      M->launches = before;
      e = cudaGraphInstantiate(&M->graph[gi], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(M, e, "graph instantiate");
    }
    CK(cudaGraphLaunch(M->graph[gi], M->stream));
    M->launches += M->graph_launches[gi];
  } else {
    if (mode == 0)
      enq_cycle64(M);
    else
      enq_cycle32(M, gi == 2);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  if (mode == 1 && M->opt.ir_fixed_point) {
    int rc = fx_recover_if_flagged(M);
    if (rc) return rc;
  }
  *norm2 = M->h_scalars[0];
  return tile_status(M);
}

int residual_norm2(hhg_mesh* M, int mode, double* norm2) {
  LevelHost& H = M->lv[M->finest];
  if (mode == 0) {
    launch_residual<double>(H.d64, M->stream);
    launch_residual_norm2<double>(H.d64, M->d_partial, M->d_scalars, M->stream);
    M->launches += 3;
  } else {
    enq_ir_residual(M, false);
    if (M->opt.ir_fixed_point)
      CK(cudaMemcpyAsync(M->h_fxmax, M->d_fxmax, sizeof(M->h_fxmax), cudaMemcpyDeviceToHost, M->stream));
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  *norm2 = M->h_scalars[0];
  return tile_status(M);
}

int check_level(hhg_mesh* M, int level) {
  if (!M) return HHG_EINVAL;
  if (level < M->coarsest || level > M->finest) return fail(M, HHG_EINVAL, "level outside the hierarchy");
  return HHG_OK;
}

// host/device pointer -> staging buffer (n * ncomp doubles)
int stage_in(hhg_mesh* M, const double* src, int64_t count) {
  CK(cudaMemcpyAsync(M->d_stage, src, sizeof(double) * (size_t)count, cudaMemcpyDefault, M->stream));
  return HHG_OK;
}
int stage_out(hhg_mesh* M, double* dst, int64_t count) {
  CK(cudaMemcpyAsync(dst, M->d_stage, sizeof(double) * (size_t)count, cudaMemcpyDefault, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return HHG_OK;
}

int do_solve(hhg_mesh* M, double tol, int max_cycles, int mode, hhg_stats* st) {
  auto t0 = std::chrono::steady_clock::now();
  if (mode == HHG_MODE_FP32_IR) {
    int rc = ensure32(M);
    if (rc) return rc;
  }
  const int64_t l0 = M->launches, x0 = M->fx_recoveries;
  double r2;
  int rc = residual_norm2(M, mode, &r2);
  if (rc) return rc;
  const double r0 = std::sqrt(r2);
  hhg_stats s{};
  s.r0 = r0;
  s.history[0] = 1.0;
  s.status = HHG_OK;
  double rel = 1.0;
  int cycles = 0;
  if (r0 > 0.0 && std::isfinite(r0)) {
    // fixed point: a field that is zero throughout has no scale for its first
    // correction, so that cycle updates in FP64 (it would be refused and redone)
    // (the velocity components share one scale: k_ir_quantize)
    const bool fp64_first = mode == HHG_MODE_FP32_IR && M->opt.ir_fixed_point &&
                            (std::max(std::max(M->h_fxmax[0], M->h_fxmax[1]), M->h_fxmax[2]) == 0 ||
                             M->h_fxmax[3] == 0);
    while (cycles < max_cycles) {
      rc = run_cycle(M, mode, &r2, cycles == 0 && fp64_first);
      if (rc) return rc;
      ++cycles;
      rel = std::sqrt(r2) / r0;
      if (cycles < 64) s.history[cycles] = rel;
      if (!std::isfinite(rel) || rel > 1e3) {
        s.status = HHG_EDIVERGED;
        break;
      }
      if (rel <= tol) break;
    }
    if (s.status == HHG_OK && rel > tol) s.status = HHG_EMAXIT;
  } else if (!std::isfinite(r0)) {
    s.status = HHG_EDIVERGED;
  }
  if (mode == HHG_MODE_FP32_IR && M->opt.ir_fixed_point && cycles > 0) fx_materialize(M);
  if (mode == HHG_MODE_FP32_IR && !M->macro.has_outflow) {
    enq_project<double>(M, M->finest);
    CK(cudaGetLastError());
  }
  s.cycles = cycles;
  s.rel_residual = rel;
  s.kernel_launches = M->launches - l0;
  s.fx_rescales = (int32_t)(M->fx_recoveries - x0);
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = s;
  if (s.status == HHG_EDIVERGED) return fail(M, HHG_EDIVERGED, "residual diverged");
  return s.status;
}

int gather_solution(hhg_mesh* M, double* u_out, double* p_out) {
  LevelHost& H = M->lv[M->finest];
  const int64_t n = H.sh.n();
  if (u_out) {
    const double* src[3] = {H.d64.u[0], H.d64.u[1], H.d64.u[2]};
    launch_gather<double>(H.d64, src, 3, M->d_stage, M->stream);
    launch_dirichlet_fill(M->d_dir_lat, M->d_dir_val, M->ndir, H.d64, M->d_stage, M->stream);
    CK(cudaGetLastError());
    int rc = stage_out(M, u_out, 3 * n);
    if (rc) return rc;
  }
  if (p_out) {
    const double* src[1] = {H.d64.p};
    launch_gather<double>(H.d64, src, 1, M->d_stage, M->stream);
    CK(cudaGetLastError());
    int rc = stage_out(M, p_out, n);
    if (rc) return rc;
  }
  return HHG_OK;
}

void release(hhg_mesh* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  for (auto& g : M->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& H : M->lv) {
    cudaFree(H.d_flags);
    cudaFree(H.d_cls);
    cudaFree(H.d_wt64);
    cudaFree(H.d_wt32);
    cudaFree(H.d_wt2_64);
    cudaFree(H.d_wt2_32);
    cudaFree(H.d_list);
    cudaFree(H.d_dir_lat);
    cudaFree(H.d_dir_pad);
    cudaFree(H.d_dir_val);
    cudaFree(H.d_irr);
    cudaFree(H.mem64);
    cudaFree(H.mem32);
  }
  cudaFree(M->d_mmask);
  cudaFree(M->d_stage);
  cudaFree(M->d_partial);
  cudaFree(M->d_ir_partial);
  cudaFree(M->d_scalars);
  cudaFree(M->d_coarse);
  cudaFree(M->d_fx);
  cudaFree(M->d_fxmax);
  cudaFree(M->d_rhs_fx);
  cudaFree(M->d_coarse_sys);
  cudaFree(M->d_backup);
  if (M->h_scalars) cudaFreeHost(M->h_scalars);
  if (M->own_stream && M->stream) cudaStreamDestroy(M->stream);
}

}  // namespace

// =============================== C ABI ==========================================

extern "C" {

void hhg_default_options(hhg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->nu = 1.0;
  opt->delta = 1.0 / 12.0;
  opt->omega = 0.3;
  opt->nu_pre = 3;
  opt->nu_post = 3;
  opt->var_increment = 2;
  opt->coarsest_level = 2;
  opt->coarse_minres_max = 5;
  opt->coarse_minres_rtol = 5e-3;
  opt->coarse_cg_max = 50;
  opt->coarse_cg_rtol = 1e-3;
  opt->use_graphs = 1;
  opt->fuse_coarse_levels = 2;
  opt->ir_fixed_point = 1;
}

const char* hhg_strerror(int code) {
  switch (code) {
    case HHG_OK: return "ok";
    case HHG_EINVAL: return "invalid argument";
    case HHG_EMESH: return "macro mesh not supported";
    case HHG_ENOMEM: return "out of device memory";
    case HHG_EDIVERGED: return "solver diverged";
    case HHG_EMAXIT: return "tolerance not reached within max_cycles";
    case HHG_ECUDA: return "CUDA error";
    case HHG_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* hhg_last_error(const hhg_mesh* mesh) {
  return mesh ? mesh->err.c_str() : g_create_error.c_str();
}

int hhg_lattice_classify(const double* V, int64_t nv, const int32_t* T, int64_t nt, const uint8_t* bc,
                         int32_t level, int64_t dims[3], uint8_t* flags) {
  if (!dims || level < 0 || level > 12) return HHG_EINVAL;
  MacroLattice m;
  int rc = build_macro_lattice(V, nv, T, nt, bc, m, g_create_error);
  if (rc) return rc;
  LevelShape sh = level_shape(m, level);
  dims[0] = sh.nx;
  dims[1] = sh.ny;
  dims[2] = sh.nz;
  if (flags) classify_nodes(m, level, flags);
  return HHG_OK;
}

int hhg_assemble_operator_host(const double* V, int64_t nv, const int32_t* T, int64_t nt, const uint8_t* bc,
                               int32_t level, const hhg_options* opt, int64_t sizes[3], int32_t* kptr,
                               int32_t* kcol, double* kval, int64_t* vnode, int64_t* pnode, double* pmass) {
  if (!sizes || level < 0 || level > 12) {
    g_create_error = "invalid level or sizes";
    return HHG_EINVAL;
  }
  hhg_options o;
  if (opt)
    o = *opt;
  else
    hhg_default_options(&o);
  if (o.nu <= 0 || o.delta <= 0 || (o.operator_form != 0 && o.operator_form != 1)) {
    g_create_error = "invalid option";
    return HHG_EINVAL;
  }
  MacroLattice m;
  int rc = build_macro_lattice(V, nv, T, nt, bc, m, g_create_error);
  if (rc) return rc;
  const LevelShape sh = level_shape(m, level);
  std::vector<uint8_t> flags(sh.n());
  classify_nodes(m, level, flags.data());
  std::vector<uint16_t> cls;
  std::vector<double> table, table2;
  std::vector<uint32_t> patterns;
  std::string err;
  int ncls = 0;
  stencil_classes(m, level, flags.data(), cls, table, ncls, err, &patterns);
  if (!err.empty()) {
    g_create_error = err;
    return HHG_EMESH;
  }
  if (o.operator_form == 1) stencil_classes_d(m, patterns, table2);
  // the scale factors of the level, as hhg_create_mesh sets them
  const double h = m.H / (double)(1 << level);
  const double hT2 = std::pow(m.det * h * h * h / 6.0, 2.0 / 3.0);
  const int64_t px = ((sh.nx + 2 + 15) / 16) * 16, pxy = px * (sh.ny + 2);
  CoarseMatrix cm;
  if ((rc = assemble_coarse(sh, px, pxy, flags.data(), cls.data(), table.data(), o.nu * h, o.delta * hT2 * h, h * h,
                            h * h * h, cm, err, o.operator_form == 1 ? table2.data() : nullptr))) {
    g_create_error = err;
    return rc;
  }
  sizes[0] = (int64_t)cm.kptr.size() - 1;
  sizes[1] = (int64_t)cm.kcol.size();
  sizes[2] = cm.nv;
  if (!kptr) return HHG_OK;
  if (!kcol || !kval || !vnode || !pnode) {
    g_create_error = "null output array";
    return HHG_EINVAL;
  }
  std::copy(cm.kptr.begin(), cm.kptr.end(), kptr);
  std::copy(cm.kcol.begin(), cm.kcol.end(), kcol);
  std::copy(cm.kval.begin(), cm.kval.end(), kval);
  // padded positions back to lattice indices
  std::vector<int64_t> lat_of((size_t)pxy * (sh.nz + 2), -1);
  for (int k = 0; k < sh.nz; ++k)
    for (int j = 0; j < sh.ny; ++j)
      for (int i = 0; i < sh.nx; ++i)
        lat_of[pad_index(px, pxy, i, j, k)] = i + (int64_t)sh.nx * (j + (int64_t)sh.ny * k);
  for (int32_t r = 0; r < cm.nv; ++r) vnode[r] = lat_of[cm.vidx[r]];
  for (int32_t r = 0; r < cm.np; ++r) pnode[r] = lat_of[cm.pidx[r]];
  if (pmass) std::copy(cm.mass.begin(), cm.mass.end(), pmass);
  return HHG_OK;
}

int hhg_create_mesh(const double* V, int64_t nv, const int32_t* T, int64_t nt, const uint8_t* bc,
                    int32_t finest, const hhg_options* opt, void* stream, hhg_mesh** out) {
  if (!out) return HHG_EINVAL;
  *out = nullptr;
  hhg_options o;
  if (opt)
    o = *opt;
  else
    hhg_default_options(&o);
  if (finest < 0 || finest > 12 || o.coarsest_level < 0 || o.coarsest_level > finest || o.nu <= 0 ||
      o.delta <= 0 || o.omega <= 0 || o.nu_pre < 0 || o.nu_post < 0 || o.var_increment < 0 ||
      o.coarse_minres_max < 0 || o.coarse_cg_max < 0) {
    g_create_error = "invalid level or option";
    return HHG_EINVAL;
  }
  if (o.operator_form != 0 && o.operator_form != 1) {
    g_create_error = "operator_form must be 0 (Laplace) or 1 (D)";
    return HHG_EINVAL;
  }
  if (o.operator_form == 1) {
    // the cluster-resident and fused levels, the fused and pair colour
    // kernels and the fixed-point refinement residual evaluate the Laplace
    // form's closed-form stencils: the D form runs the per-level kernels with
    // its class rows and the FP64 refinement residual
    o.fuse_coarse_levels = 0;
    o.ir_fixed_point = 0;
    o.fused_min_nodes = -1;
    o.colour_pairs = -1;
  }
  hhg_mesh* M = new hhg_mesh();
  M->opt = o;
  M->finest = finest;
  M->coarsest = o.coarsest_level;
  int rc = build_macro_lattice(V, nv, T, nt, bc, M->macro, g_create_error);
  if (rc) {
    delete M;
    return rc;
  }
  auto bail = [&](int code) {
    g_create_error = M->err;
    release(M);
    delete M;
    return code;
  };
  cudaError_t e = cudaGetDevice(&M->device);
  if (e != cudaSuccess) {
    M->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return bail(HHG_ECUDA);
  }
  if (stream) {
    M->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      M->err = std::string("stream: ") + cudaGetErrorString(e);
      return bail(HHG_ECUDA);
    }
    M->own_stream = true;
  }
  if ((rc = dalloc(M, (void**)&M->d_mmask, M->macro.mask.size()))) return bail(rc);
  if ((e = cudaMemcpy(M->d_mmask, M->macro.mask.data(), M->macro.mask.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    M->err = cudaGetErrorString(e);
    return bail(HHG_ECUDA);
  }
  M->lv.resize(finest + 1);
  for (int l = M->coarsest; l <= finest; ++l) {
    LevelHost& H = M->lv[l];
    H.level = l;
    H.sh = level_shape(M->macro, l);
    H.px = ((H.sh.nx + 2 + 15) / 16) * 16;  // rows grouped by x mod 4 (hhg_common.h), 16-byte aligned groups
    H.py = H.sh.ny + 2;
    H.pz = H.sh.nz + 2;
    H.nalloc = H.px * H.py * H.pz;
    H.h = M->macro.H / (double)(1 << l);
    // h_T = |T|^(1/3), |T| = det h^3 / 6 (det = 1 on axis-aligned lattices)
    H.hT2 = std::pow(M->macro.det * H.h * H.h * H.h / 6.0, 2.0 / 3.0);
    H.flags.resize(H.sh.n());
    classify_nodes(M->macro, l, H.flags.data());
    std::vector<uint8_t> padded(H.nalloc, 0);
    for (int k = 0; k < H.sh.nz; ++k)
      for (int j = 0; j < H.sh.ny; ++j)
        for (int i = 0; i < H.sh.nx; ++i) {
          const uint8_t f = H.flags[i + (int64_t)H.sh.nx * (j + (int64_t)H.sh.ny * k)];
          padded[pad_index(H.px, H.px * H.py, i, j, k)] = f;
          if (f & F_VFREE) H.n_vel++;
          if (f & F_ACT) H.n_pres++;
        }
    if ((rc = dalloc(M, (void**)&H.d_flags, H.nalloc))) return bail(rc);
    if ((e = cudaMemcpy(H.d_flags, padded.data(), H.nalloc, cudaMemcpyHostToDevice)) != cudaSuccess) {
      M->err = cudaGetErrorString(e);
      return bail(HHG_ECUDA);
    }
    // stencil classes of the boundary nodes and their row tables
    {
      std::vector<uint16_t> cls;
      std::vector<double> table;
      std::vector<uint32_t> patterns;
      std::string cerr;
      stencil_classes(M->macro, l, H.flags.data(), cls, table, H.n_classes, cerr, &patterns);
      if (!cerr.empty()) {
        M->err = cerr;
        return bail(HHG_EMESH);
      }
      if (o.operator_form == 1) {
        std::vector<double> table2;
        stencil_classes_d(M->macro, patterns, table2);
        std::vector<float> table2_32(table2.begin(), table2.end());
        if ((rc = dalloc(M, (void**)&H.d_wt2_64, sizeof(double) * table2.size()))) return bail(rc);
        if ((rc = dalloc(M, (void**)&H.d_wt2_32, sizeof(float) * table2.size()))) return bail(rc);
        if (cudaMemcpy(H.d_wt2_64, table2.data(), sizeof(double) * table2.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(H.d_wt2_32, table2_32.data(), sizeof(float) * table2.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
          M->err = "upload of the D-form stencil tables failed";
          return bail(HHG_ECUDA);
        }
      }
      std::vector<uint16_t> pcls(H.nalloc, 0);
      for (int k = 0; k < H.sh.nz; ++k)
        for (int j = 0; j < H.sh.ny; ++j)
          for (int i = 0; i < H.sh.nx; ++i)
            pcls[pad_index(H.px, H.px * H.py, i, j, k)] =
                cls[i + (int64_t)H.sh.nx * (j + (int64_t)H.sh.ny * k)];
      std::vector<float> table32(table.begin(), table.end());
      if ((rc = dalloc(M, (void**)&H.d_cls, sizeof(uint16_t) * (size_t)H.nalloc))) return bail(rc);
      if ((rc = dalloc(M, (void**)&H.d_wt64, sizeof(double) * table.size()))) return bail(rc);
      if ((rc = dalloc(M, (void**)&H.d_wt32, sizeof(float) * table.size()))) return bail(rc);
      if (cudaMemcpy(H.d_cls, pcls.data(), sizeof(uint16_t) * pcls.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(H.d_wt64, table.data(), sizeof(double) * table.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(H.d_wt32, table32.data(), sizeof(float) * table32.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        M->err = "upload of stencil tables failed";
        return bail(HHG_ECUDA);
      }
    }
    if ((rc = dalloc(M, (void**)&H.mem64, sizeof(double) * 12 * (size_t)H.nalloc))) return bail(rc);
    if ((e = cudaMemset(H.mem64, 0, sizeof(double) * 12 * (size_t)H.nalloc)) != cudaSuccess) {
      M->err = cudaGetErrorString(e);
      return bail(HHG_ECUDA);
    }
    bind_fields(H.d64, H.mem64, H.nalloc);
    fill_coefs(M, H);
  }
  // Dirichlet nodes and boundary (F_IRR) nodes of every level (compact lists)
  for (int l = M->coarsest; l <= finest; ++l) {
    LevelHost& H = M->lv[l];
    std::vector<int64_t> lat, pad, irr;
    for (int64_t k = 0; k < H.sh.nz; ++k)
      for (int64_t j = 0; j < H.sh.ny; ++j)
        for (int64_t i = 0; i < H.sh.nx; ++i) {
          const int64_t q = i + H.sh.nx * (j + H.sh.ny * k);
          const uint8_t f = H.flags[q];
          if ((f & F_DIR) && (f & F_ACT)) {
            lat.push_back(q);
            pad.push_back(pad_index(H.px, H.px * H.py, (int)i, (int)j, (int)k));
          }
          if (f & F_IRR) irr.push_back((k << 42) | (j << 21) | i);
        }
    H.ndir = (int64_t)lat.size();
    if (H.ndir) {
      if ((rc = dalloc(M, (void**)&H.d_dir_lat, sizeof(int64_t) * lat.size()))) return bail(rc);
      if ((rc = dalloc(M, (void**)&H.d_dir_pad, sizeof(int64_t) * pad.size()))) return bail(rc);
      if ((rc = dalloc(M, (void**)&H.d_dir_val, sizeof(double) * 3 * lat.size()))) return bail(rc);
      cudaMemcpy(H.d_dir_lat, lat.data(), sizeof(int64_t) * lat.size(), cudaMemcpyHostToDevice);
      cudaMemcpy(H.d_dir_pad, pad.data(), sizeof(int64_t) * pad.size(), cudaMemcpyHostToDevice);
      cudaMemset(H.d_dir_val, 0, sizeof(double) * 3 * lat.size());
    }
    H.nirr = (int64_t)irr.size();
    if ((rc = dalloc(M, (void**)&H.d_irr, sizeof(int64_t) * std::max<size_t>(irr.size(), 1)))) return bail(rc);
    if (!irr.empty() &&
        (e = cudaMemcpy(H.d_irr, irr.data(), sizeof(int64_t) * irr.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
      M->err = std::string("set-up: ") + cudaGetErrorString(e);
      return bail(HHG_ECUDA);
    }
  }
  {
    LevelHost& H = M->lv[finest];
    M->ndir = H.ndir;
    M->d_dir_lat = H.d_dir_lat;
    M->d_dir_pad = H.d_dir_pad;
    M->d_dir_val = H.d_dir_val;
    M->n_fx_irr = H.nirr;
    M->d_fx_irr = H.d_irr;
    if ((rc = dalloc(M, (void**)&M->d_stage, sizeof(double) * 3 * (size_t)H.sh.n()))) return bail(rc);
  }
  if ((rc = dalloc(M, (void**)&M->d_partial, sizeof(double) * 4 * std::max(REDUCE_BLOCKS, IR_BLOCKS + IR_IRR_BLOCKS)))) return bail(rc);
  if ((rc = dalloc(M, (void**)&M->d_ir_partial, sizeof(double) * ir_residual_fx_partials(M->lv[finest].d64))))
    return bail(rc);
  if ((rc = dalloc(M, (void**)&M->d_scalars, sizeof(double) * 16))) return bail(rc);
  cudaMemset(M->d_scalars, 0, sizeof(double) * 16);
  if ((rc = dalloc(M, (void**)&M->d_rhs_fx, sizeof(unsigned long long) * 10))) return bail(rc);
  if ((e = cudaMallocHost((void**)&M->h_scalars, sizeof(double) * 16)) != cudaSuccess) {
    M->err = cudaGetErrorString(e);
    return bail(HHG_ENOMEM);
  }
  M->allocations += 1;
  // compact coarsest-level system for the coarse solver
  {
    LevelHost& H = M->lv[M->coarsest];
    std::vector<uint16_t> cls;
    std::vector<double> table, table2;
    std::vector<uint32_t> patterns;
    std::string cerr;
    int ncls = 0;
    stencil_classes(M->macro, H.level, H.flags.data(), cls, table, ncls, cerr, &patterns);
    if (o.operator_form == 1) stencil_classes_d(M->macro, patterns, table2);
    CoarseMatrix cm;
    if (cerr.empty() &&
        (rc = assemble_coarse(H.sh, H.px, H.px * H.py, H.flags.data(), cls.data(), table.data(), H.d64.nuh, H.d64.c,
                              H.d64.h2, H.d64.h3, cm, cerr, o.operator_form == 1 ? table2.data() : nullptr))) {
      M->err = cerr;
      return bail(rc);
    }
    if (!cerr.empty()) {
      M->err = cerr;
      return bail(HHG_EMESH);
    }
    // one allocation, 8-byte aligned parts: doubles first, then the indices
    const size_t nd = cm.kval.size() + cm.aval.size() + cm.mass.size();
    const size_t ni = cm.vidx.size() + cm.pidx.size() + cm.kptr.size() + cm.kcol.size() + cm.aptr.size() +
                      cm.acol.size();
    if ((rc = dalloc(M, &M->d_coarse_sys, sizeof(double) * nd + sizeof(int32_t) * ni + 16))) return bail(rc);
    double* dp = (double*)M->d_coarse_sys;
    int32_t* ip = (int32_t*)(dp + nd);
    auto put_d = [&](const std::vector<double>& v) {
      double* at = dp;
      if (!v.empty()) cudaMemcpy(at, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
      dp += v.size();
      return at;
    };
    auto put_i = [&](const std::vector<int32_t>& v) {
      int32_t* at = ip;
      if (!v.empty()) cudaMemcpy(at, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
      ip += v.size();
      return at;
    };
    CoarseSys& S = M->coarse_sys;
    S.nv = cm.nv;
    S.np = cm.np;
    S.coupled = cm.coupled;
    S.kval = put_d(cm.kval);
    S.aval = put_d(cm.aval);
    S.mass = put_d(cm.mass);
    S.vidx = put_i(cm.vidx);
    S.pidx = put_i(cm.pidx);
    S.kptr = put_i(cm.kptr);
    S.kcol = put_i(cm.kcol);
    S.aptr = put_i(cm.aptr);
    S.acol = put_i(cm.acol);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      M->err = std::string("upload of the coarse system: ") + cudaGetErrorString(e);
      return bail(HHG_ECUDA);
    }
  }
  if ((rc = dalloc(M, (void**)&M->d_coarse, sizeof(double) * (size_t)std::max<int64_t>(1, coarse_scratch_doubles(M->coarse_sys)))))
    return bail(rc);
  // colour-fused FP32 passes on the large levels (planned when the FP32 fields are allocated)
  prepare_fused();
  // cluster kernels (fused coarse levels, coarse solve)
  prepare_coarse_solve();
  {
    const unsigned cl = prepare_small_cycle();
    M->small_cluster[0] = o.team_blocks > 0 ? std::min<unsigned>((unsigned)o.team_blocks, cl) : SMALL_TEAM_BLOCKS_FP64;
    M->small_cluster[1] = o.team_blocks > 0 ? std::min<unsigned>((unsigned)o.team_blocks, cl)
                                            : std::min<unsigned>(SMALL_TEAM_BLOCKS, cl);
  }
  // cluster-resident coarse levels: the largest level whose sub-hierarchy fits
  // the shared memory of one cluster (and has at most fuse_max_nodes nodes)
  if (o.fuse_coarse_levels == 2) {
    const int64_t lim = o.fuse_max_nodes > 0 ? o.fuse_max_nodes : RES_MAX_NODES;
    if (o.resident_node_lists >= 0)
      for (int l = M->coarsest + 1; l <= std::min(finest, M->coarsest + RES_MAX_LEVELS); ++l)
        if (M->lv[l].sh.n() <= lim && (rc = build_node_lists(M, M->lv[l]))) return bail(rc);
    for (int pr = 0; pr < 2; ++pr) {
      M->res_nb[pr] = pr ? prepare_resident<float>(M->res_smem[pr]) : prepare_resident<double>(M->res_smem[pr]);
      const unsigned want = o.team_blocks > 0 ? (unsigned)o.team_blocks : (pr ? RES_CTAS_FP32 : RES_CTAS_FP64);
      M->res_nb[pr] = std::min<unsigned>(M->res_nb[pr], want);
      for (int l = std::min(finest, M->coarsest + RES_MAX_LEVELS); l > M->coarsest; --l) {
        if (M->lv[l].sh.n() > lim) continue;
        bool fits;
        if (pr) {
          ResidentCycle<float> S;
          fill_resident<float>(M, S, l);
          fits = plan_resident<float>(S, M->res_smem[pr], M->res_nb[pr]);
        } else {
          ResidentCycle<double> S;
          fill_resident<double>(M, S, l);
          fits = plan_resident<double>(S, M->res_smem[pr], M->res_nb[pr]);
        }
        if (fits) {
          M->res_top[pr] = l;
          break;
        }
      }
    }
  }
  // fused coarse levels: the largest level of at most fuse_max_nodes nodes
  if (o.fuse_coarse_levels == 1 || (o.fuse_coarse_levels == 2 && (M->res_top[0] < 0 || M->res_top[1] < 0))) {
    const int64_t lim32 = o.fuse_max_nodes > 0 ? o.fuse_max_nodes : SMALL_MAX_NODES;
    const int64_t lim64 = o.fuse_max_nodes > 0 ? o.fuse_max_nodes : SMALL_MAX_NODES_FP64;
    for (int l = M->coarsest + 1; l <= finest && l - M->coarsest < SMALL_MAX_LEVELS; ++l) {
      if (M->lv[l].sh.n() <= lim64) M->small_top[0] = l;
      if (M->lv[l].sh.n() <= lim32) M->small_top[1] = l;
    }
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    M->err = std::string("set-up: ") + cudaGetErrorString(e);
    return bail(HHG_ECUDA);
  }
  *out = M;
  return HHG_OK;
}

void hhg_destroy(hhg_mesh* mesh) {
  if (!mesh) return;
  release(mesh);
  delete mesh;
}

int hhg_lattice_dims(const hhg_mesh* mesh, int32_t level, int64_t dims[3]) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!dims) return HHG_EINVAL;
  dims[0] = M->lv[level].sh.nx;
  dims[1] = M->lv[level].sh.ny;
  dims[2] = M->lv[level].sh.nz;
  return HHG_OK;
}

int hhg_num_nodes(const hhg_mesh* mesh, int32_t level, int64_t* n) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!n) return HHG_EINVAL;
  *n = M->lv[level].sh.n();
  return HHG_OK;
}

int hhg_num_dofs(const hhg_mesh* mesh, int32_t level, int64_t* nv, int64_t* np) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (nv) *nv = M->lv[level].n_vel;
  if (np) *np = M->lv[level].n_pres;
  return HHG_OK;
}

int hhg_node_coords(const hhg_mesh* mesh, int32_t level, double* xyz) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!xyz) return HHG_EINVAL;
  const LevelHost& H = M->lv[level];
  std::vector<double> tmp(3 * (size_t)H.sh.n());
  for (int k = 0; k < H.sh.nz; ++k)
    for (int j = 0; j < H.sh.ny; ++j)
      for (int i = 0; i < H.sh.nx; ++i) {
        const int64_t q = i + (int64_t)H.sh.nx * (j + (int64_t)H.sh.ny * k);
        const double* B0 = M->macro.basis[0];
        const double* B1 = M->macro.basis[1];
        const double* B2 = M->macro.basis[2];
        tmp[3 * q + 0] = M->macro.origin[0] + H.h * (B0[0] * i + B0[1] * j + B0[2] * k);
        tmp[3 * q + 1] = M->macro.origin[1] + H.h * (B1[0] * i + B1[1] * j + B1[2] * k);
        tmp[3 * q + 2] = M->macro.origin[2] + H.h * (B2[0] * i + B2[1] * j + B2[2] * k);
      }
  CK(cudaMemcpy(xyz, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyDefault));
  return HHG_OK;
}

int hhg_node_flags(const hhg_mesh* mesh, int32_t level, uint8_t* flags) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!flags) return HHG_EINVAL;
  CK(cudaMemcpy(flags, M->lv[level].flags.data(), M->lv[level].flags.size(), cudaMemcpyDefault));
  return HHG_OK;
}

int hhg_outflow_weights(const hhg_mesh* mesh, int32_t level, double* w) {
  hhg_mesh* M = const_cast<hhg_mesh*>(mesh);
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!w) return HHG_EINVAL;
  std::vector<double> tmp(3 * (size_t)M->lv[level].sh.n());
  outflow_weights(M->macro, level, tmp.data());
  CK(cudaMemcpy(w, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyDefault));
  return HHG_OK;
}

int hhg_device_bytes(const hhg_mesh* mesh, int64_t* bytes) {
  if (!mesh || !bytes) return HHG_EINVAL;
  *bytes = mesh->device_bytes;
  return HHG_OK;
}

int hhg_set_rhs(hhg_mesh* M, const double* f_nodal, const double* u_dirichlet) {
  if (!M) return HHG_EINVAL;
  CK(cudaSetDevice(M->device));
  LevelHost& H = M->lv[M->finest];
  LevelDev<double>& L = H.d64;
  const int64_t n = H.sh.n();
  launch_zero<double>(L, 0, M->stream);
  launch_zero<double>(L, 2, M->stream);
  // staged body force in RU (active nodes), Dirichlet data in U (Dirichlet nodes)
  if (f_nodal) {
    int rc = stage_in(M, f_nodal, 3 * n);
    if (rc) return rc;
    launch_scatter(L, M->d_stage, 3, L.r, F_ACT, M->stream);
  }
  if (u_dirichlet) {
    int rc = stage_in(M, u_dirichlet, 3 * n);
    if (rc) return rc;
    launch_scatter(L, M->d_stage, 3, L.u, F_DIR, M->stream);
  }
  launch_dirichlet_gather(M->d_dir_pad, M->ndir, L, M->d_dir_val, M->stream);  // before U is quantized
  launch_set_rhs(L, L.r, L.u, M->d_rhs_fx, reinterpret_cast<int*>(M->d_rhs_fx + 8), M->d_fx_irr, M->n_fx_irr,
                 M->stream);
  if (L.wt2) {
    launch_lift_d(L, L.u, reinterpret_cast<const int*>(M->d_rhs_fx + 8), M->stream);
    M->launches += 1;
  }
  if (!M->macro.has_outflow) launch_remove_mean_g(L, M->d_partial, M->d_scalars + 3, M->stream);
  M->launches += (f_nodal ? 1 : 0) + (u_dirichlet ? 1 : 0) + 4 + (M->n_fx_irr ? 1 : 0) +
                 (M->macro.has_outflow ? 0 : 3) + (M->ndir ? 1 : 0);
  launch_zero<double>(L, 0, M->stream);
  launch_zero<double>(L, 2, M->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(M->stream));
  M->rhs_set = true;
  return HHG_OK;
}

int hhg_set_initial(hhg_mesh* M, const double* u, const double* p) {
  if (!M) return HHG_EINVAL;
  if (!M->rhs_set) return fail(M, HHG_ESTATE, "hhg_set_initial before hhg_set_rhs");
  CK(cudaSetDevice(M->device));
  LevelHost& H = M->lv[M->finest];
  LevelDev<double>& L = H.d64;
  const int64_t n = H.sh.n();
  launch_zero<double>(L, 0, M->stream);
  if (u) {
    int rc = stage_in(M, u, 3 * n);
    if (rc) return rc;
    launch_scatter(L, M->d_stage, 3, L.u, F_VFREE, M->stream);
    enq_slip_fix(M, M->finest, false);  // a free-slip node's velocity is tangential
  }
  if (p) {
    int rc = stage_in(M, p, n);
    if (rc) return rc;
    double* dst[1] = {L.p};
    launch_scatter(L, M->d_stage, 1, dst, F_ACT, M->stream);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(M->stream));
  return HHG_OK;
}

int hhg_vcycle(hhg_mesh* M, int32_t count, double* rel) {
  if (!M || count < 0) return HHG_EINVAL;
  if (!M->rhs_set) return fail(M, HHG_ESTATE, "hhg_vcycle before hhg_set_rhs");
  CK(cudaSetDevice(M->device));
  double r2;
  int rc = residual_norm2(M, 0, &r2);
  if (rc) return rc;
  const double r0 = std::sqrt(r2);
  double cur = r2;
  for (int c = 0; c < count; ++c) {
    rc = run_cycle(M, 0, &cur);
    if (rc) return rc;
  }
  if (rel) *rel = r0 > 0 ? std::sqrt(cur) / r0 : 0.0;
  return HHG_OK;
}

int hhg_solve(hhg_mesh* M, double tol, int32_t max_cycles, int32_t mode, double* u_out, double* p_out,
              hhg_stats* stats) {
  if (!M || max_cycles < 0 || !(tol >= 0) || (mode != HHG_MODE_FP64 && mode != HHG_MODE_FP32_IR))
    return HHG_EINVAL;
  if (!M->rhs_set) return fail(M, HHG_ESTATE, "hhg_solve before hhg_set_rhs");
  CK(cudaSetDevice(M->device));
  int rc = do_solve(M, tol, max_cycles, mode, stats);
  if (rc != HHG_OK && rc != HHG_EMAXIT) return rc;
  int rc2 = gather_solution(M, u_out, p_out);
  return rc2 ? rc2 : rc;
}

int hhg_fmg_solve(hhg_mesh* M, const double* f_nodal, const double* u_dirichlet, int32_t cycles, int32_t nu,
                  int32_t mode, double* u_out, double* p_out, hhg_stats* stats) {
  if (!M || cycles < 0 || nu < 0 || (mode != HHG_MODE_FP64 && mode != HHG_MODE_FP32_IR)) return HHG_EINVAL;
  CK(cudaSetDevice(M->device));
  if (mode == HHG_MODE_FP32_IR) {
    int rc = ensure32(M);
    if (rc) return rc;
  }
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = M->launches;
  LevelHost& Fh = M->lv[M->finest];
  LevelDev<double>& Lf = Fh.d64;
  const int64_t n = Fh.sh.n();
  for (int l = M->coarsest; l <= M->finest; ++l) {
    launch_zero<double>(M->lv[l].d64, 0, M->stream);
    launch_zero<double>(M->lv[l].d64, 2, M->stream);
  }
  // nodal data staged as hhg_set_rhs does: body force in RU, Dirichlet data in U
  if (f_nodal) {
    int rc = stage_in(M, f_nodal, 3 * n);
    if (rc) return rc;
    launch_scatter(Lf, M->d_stage, 3, Lf.r, F_ACT, M->stream);
  }
  if (u_dirichlet) {
    int rc = stage_in(M, u_dirichlet, 3 * n);
    if (rc) return rc;
    launch_scatter(Lf, M->d_stage, 3, Lf.u, F_DIR, M->stream);
  }
  // right-hand side rediscretised on every level (Sec. 2.1 forms with the
  // data at that level's nodes); the finest level's staged data, the source
  // of the coarser levels', is quantized last
  for (int l = M->coarsest; l <= M->finest; ++l) {
    LevelHost& H = M->lv[l];
    LevelDev<double>& L = H.d64;
    if (l < M->finest) launch_inject(Lf, L, 1 << (M->finest - l), M->stream);
    launch_dirichlet_gather(H.d_dir_pad, H.ndir, L, H.d_dir_val, M->stream);
    launch_set_rhs(L, L.r, L.u, M->d_rhs_fx, reinterpret_cast<int*>(M->d_rhs_fx + 8), H.d_irr, H.nirr, M->stream);
    if (L.wt2) {
      launch_lift_d(L, L.u, reinterpret_cast<const int*>(M->d_rhs_fx + 8), M->stream);
      M->launches += 1;
    }
    if (!M->macro.has_outflow) launch_remove_mean_g(L, M->d_partial, M->d_scalars + 3, M->stream);
    launch_zero<double>(L, 0, M->stream);
    launch_zero<double>(L, 2, M->stream);
    M->launches += (l < M->finest ? 1 : 0) + (H.ndir ? 1 : 0) + 4 + (H.nirr ? 1 : 0) +
                   (M->macro.has_outflow ? 0 : 3);
  }
  M->launches += (f_nodal ? 1 : 0) + (u_dirichlet ? 1 : 0);
  M->rhs_set = true;
  double r2;
  int rc = residual_norm2(M, 0, &r2);  // of the zero iterate: ||f~||
  if (rc) return rc;
  const double r0 = std::sqrt(r2);
  // coarsest level: the coarse solver from zero; then, level by level, the P1
  // interpolant of the coarser solution (its Dirichlet values included) and
  // `cycles` V_var(nu, nu) cycles rooted at the level (Sec. 5)
  M->vnu = nu;
  M->vroot = M->coarsest;
  enq_vcycle<double>(M, M->coarsest);
  if (!M->macro.has_outflow) enq_project<double>(M, M->coarsest);
  int ncyc = 0;
  for (int l = M->coarsest + 1; l <= M->finest; ++l) {
    LevelHost& C = M->lv[l - 1];
    launch_dirichlet_scatter(C.d_dir_pad, C.ndir, C.d_dir_val, C.d64, M->stream);
    launch_prolong_add<double>(M->lv[l].d64, C.d64, M->stream);
    M->launches += (C.ndir ? 1 : 0) + 1;
    M->vroot = l;
    LevelHost& H = M->lv[l];
    for (int c = 0; c < cycles; ++c, ++ncyc) {
      if (mode == HHG_MODE_FP64) {
        enq_vcycle<double>(M, l);
      } else {
        // FP32 correction cycle from zero on the FP64 residual, FP64 update
        launch_zero<float>(H.d32, 0, M->stream);
        launch_ir_residual(H.d64, H.d32, M->d_partial, M->d_scalars, M->stream);
        enq_vcycle<float>(M, l);
        launch_ir_update(H.d64, H.d32, M->stream);
        M->launches += 3;
        enq_slip_fix(M, l, false);
      }
      if (!M->macro.has_outflow) enq_project<double>(M, l);
    }
  }
  M->vroot = -1;
  M->vnu = -1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(M, e, "fmg");
  rc = residual_norm2(M, 0, &r2);
  if (rc) return rc;
  hhg_stats s{};
  s.cycles = ncyc;
  s.status = HHG_OK;
  s.r0 = r0;
  s.rel_residual = r0 > 0 ? std::sqrt(r2) / r0 : 0.0;
  s.history[0] = 1.0;
  s.history[1] = s.rel_residual;
  if (!std::isfinite(s.rel_residual)) s.status = HHG_EDIVERGED;
  s.kernel_launches = M->launches - l0;
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = s;
  if (s.status == HHG_EDIVERGED) return fail(M, HHG_EDIVERGED, "FMG diverged");
  return gather_solution(M, u_out, p_out);
}

int hhg_get_solution(hhg_mesh* M, double* u_out, double* p_out) {
  if (!M) return HHG_EINVAL;
  CK(cudaSetDevice(M->device));
  return gather_solution(M, u_out, p_out);
}

int hhg_apply_operator(hhg_mesh* M, int32_t level, const double* u, const double* p, double* ku, double* kp) {
  int rc = check_level(M, level);
  if (rc) return rc;
  CK(cudaSetDevice(M->device));
  LevelHost& H = M->lv[level];
  const int64_t n = H.sh.n();
  double* tmp = nullptr;
  if ((rc = dalloc(M, (void**)&tmp, sizeof(double) * 12 * (size_t)H.nalloc))) return rc;
  M->device_bytes -= (int64_t)(sizeof(double) * 12 * (size_t)H.nalloc);
  cudaMemsetAsync(tmp, 0, sizeof(double) * 12 * (size_t)H.nalloc, M->stream);
  LevelDev<double> L = H.d64;
  bind_fields(L, tmp, H.nalloc);
  double* stage = nullptr;
  if ((rc = dalloc(M, (void**)&stage, sizeof(double) * 3 * (size_t)n))) {
    cudaFree(tmp);
    return rc;
  }
  M->device_bytes -= (int64_t)(sizeof(double) * 3 * (size_t)n);
  auto done = [&](int code) {
    cudaStreamSynchronize(M->stream);
    cudaFree(tmp);
    cudaFree(stage);
    return code;
  };
  if (u) {
    if (cudaMemcpyAsync(stage, u, sizeof(double) * 3 * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy u"));
    launch_scatter(L, stage, 3, L.u, F_VFREE, M->stream);
  }
  if (p) {
    if (cudaMemcpyAsync(stage, p, sizeof(double) * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy p"));
    double* dst[1] = {L.p};
    launch_scatter(L, stage, 1, dst, F_ACT, M->stream);
  }
  launch_residual<double>(L, M->stream);  // (RU, RP) = -K (U, P) since F = G = 0
  if (ku) {
    const double* src[3] = {L.r[0], L.r[1], L.r[2]};
    launch_gather<double>(L, src, 3, stage, M->stream);
    launch_scale(stage, 3 * n, -1.0, M->stream);
    if (cudaMemcpyAsync(ku, stage, sizeof(double) * 3 * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy ku"));
    cudaStreamSynchronize(M->stream);
  }
  if (kp) {
    const double* src[1] = {L.rp};
    launch_gather<double>(L, src, 1, stage, M->stream);
    launch_scale(stage, n, -1.0, M->stream);
    if (cudaMemcpyAsync(kp, stage, sizeof(double) * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy kp"));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_fail(M, e, "apply_operator"));
  return done(HHG_OK);
}

int hhg_adjoint_gradient(hhg_mesh* M, const double* ju, const double* jp, double tol, int32_t max_cycles,
                         int32_t mode, double* grad_f, hhg_stats* stats) {
  if (!M || !grad_f || (mode != HHG_MODE_FP64 && mode != HHG_MODE_FP32_IR)) return HHG_EINVAL;
  if (!M->macro.has_outflow) return fail(M, HHG_EINVAL, "adjoint needs a mesh with an outflow face");
  CK(cudaSetDevice(M->device));
  LevelHost& H = M->lv[M->finest];
  LevelDev<double>& L = H.d64;
  const int64_t n = H.sh.n();
  const size_t fb = sizeof(double) * 8 * (size_t)H.nalloc;
  int rc;
  if (!M->d_backup && (rc = dalloc(M, (void**)&M->d_backup, fb))) return rc;
  CK(cudaMemcpyAsync(M->d_backup, L.u[0], fb, cudaMemcpyDeviceToDevice, M->stream));  // U, P, F, G
  const bool had_rhs = M->rhs_set;
  launch_zero<double>(L, 0, M->stream);
  launch_zero<double>(L, 1, M->stream);
  if (ju) {
    if ((rc = stage_in(M, ju, 3 * n))) return rc;
    launch_scatter(L, M->d_stage, 3, L.f, F_VFREE, M->stream);
  }
  if (jp) {
    if ((rc = stage_in(M, jp, n))) return rc;
    double* dst[1] = {L.g};
    launch_scatter(L, M->d_stage, 1, dst, F_ACT, M->stream);
  }
  M->rhs_set = true;
  rc = do_solve(M, tol, max_cycles, mode, stats);
  if (rc == HHG_OK || rc == HHG_EMAXIT) {
    launch_rhs_transpose(L, L.r, M->stream);
    const double* src[3] = {L.r[0], L.r[1], L.r[2]};
    launch_gather<double>(L, src, 3, M->d_stage, M->stream);
    int rc2 = stage_out(M, grad_f, 3 * n);
    if (rc2) rc = rc2;
  }
  cudaMemcpyAsync(L.u[0], M->d_backup, fb, cudaMemcpyDeviceToDevice, M->stream);
  cudaStreamSynchronize(M->stream);
  M->rhs_set = had_rhs;
  return rc;
}

int hhg_level_field(hhg_mesh* M, int32_t level, int32_t precision, int32_t field, int32_t write, double* buf) {
  int rc = check_level(M, level);
  if (rc) return rc;
  if (!buf || field < 0 || field > 5 || (precision != 0 && precision != 1)) return fail(M, HHG_EINVAL, "bad field");
  CK(cudaSetDevice(M->device));
  if (precision == 1 && (rc = ensure32(M))) return rc;
  LevelHost& H = M->lv[level];
  const int64_t n = H.sh.n();
  const int ncomp = (field == HHG_FIELD_U || field == HHG_FIELD_F || field == HHG_FIELD_RU) ? 3 : 1;
  const uint8_t mask = (field == HHG_FIELD_U || field == HHG_FIELD_F || field == HHG_FIELD_RU) ? F_VFREE : F_ACT;
  auto ptrs64 = [&](LevelDev<double>& L, double** out) {
    switch (field) {
      case HHG_FIELD_U: out[0] = L.u[0]; out[1] = L.u[1]; out[2] = L.u[2]; break;
      case HHG_FIELD_P: out[0] = L.p; break;
      case HHG_FIELD_F: out[0] = L.f[0]; out[1] = L.f[1]; out[2] = L.f[2]; break;
      case HHG_FIELD_G: out[0] = L.g; break;
      case HHG_FIELD_RU: out[0] = L.r[0]; out[1] = L.r[1]; out[2] = L.r[2]; break;
      default: out[0] = L.rp; break;
    }
  };
  auto ptrs32 = [&](LevelDev<float>& L, float** out) {
    switch (field) {
      case HHG_FIELD_U: out[0] = L.u[0]; out[1] = L.u[1]; out[2] = L.u[2]; break;
      case HHG_FIELD_P: out[0] = L.p; break;
      case HHG_FIELD_F: out[0] = L.f[0]; out[1] = L.f[1]; out[2] = L.f[2]; break;
      case HHG_FIELD_G: out[0] = L.g; break;
      case HHG_FIELD_RU: out[0] = L.r[0]; out[1] = L.r[1]; out[2] = L.r[2]; break;
      default: out[0] = L.rp; break;
    }
  };
  double* stage = nullptr;
  if ((rc = dalloc(M, (void**)&stage, sizeof(double) * 3 * (size_t)n))) return rc;
  M->device_bytes -= (int64_t)(sizeof(double) * 3 * (size_t)n);
  double* tmp = nullptr;
  auto done = [&](int code) {
    cudaStreamSynchronize(M->stream);
    cudaFree(stage);
    cudaFree(tmp);
    return code;
  };
  if (write) {
    if (cudaMemcpyAsync(stage, buf, sizeof(double) * ncomp * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy in"));
    if (precision == 0) {
      double* dst[3];
      ptrs64(H.d64, dst);
      launch_scatter(H.d64, stage, ncomp, dst, mask, M->stream);
    } else {
      if ((rc = dalloc(M, (void**)&tmp, sizeof(double) * 3 * (size_t)H.nalloc))) return done(rc);
      M->device_bytes -= (int64_t)(sizeof(double) * 3 * (size_t)H.nalloc);
      // the scatter writes lattice nodes only: the frame and row padding must
      // reach the FP32 field as zeros, not as what the allocation held
      cudaMemsetAsync(tmp, 0, sizeof(double) * 3 * (size_t)H.nalloc, M->stream);
      double* dst[3] = {tmp, tmp + H.nalloc, tmp + 2 * H.nalloc};
      launch_scatter(H.d64, stage, ncomp, dst, mask, M->stream);
      float* d32[3];
      ptrs32(H.d32, d32);
      for (int c = 0; c < ncomp; ++c) launch_cast_field(dst[c], d32[c], H.nalloc, M->stream);
    }
  } else {
    if (precision == 0) {
      double* src[3];
      ptrs64(H.d64, src);
      const double* cs[3] = {src[0], ncomp > 1 ? src[1] : src[0], ncomp > 2 ? src[2] : src[0]};
      launch_gather<double>(H.d64, cs, ncomp, stage, M->stream);
    } else {
      float* src[3];
      ptrs32(H.d32, src);
      const float* cs[3] = {src[0], ncomp > 1 ? src[1] : src[0], ncomp > 2 ? src[2] : src[0]};
      launch_gather<float>(H.d32, cs, ncomp, stage, M->stream);
    }
    if (cudaMemcpyAsync(buf, stage, sizeof(double) * ncomp * n, cudaMemcpyDefault, M->stream) != cudaSuccess)
      return done(fail(M, HHG_ECUDA, "copy out"));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_fail(M, e, "level_field"));
  return done(HHG_OK);
}

static int enqueue_op(hhg_mesh* M, int32_t level, int32_t precision, int32_t op);

int hhg_coarse_solve_noalloc(hhg_mesh* M, const double* f, const double* g, double* u, double* p) {
  if (!M || !f || !g || !u || !p) return HHG_EINVAL;
  // size check before anything is staged: a rejected call writes nothing
  if (coarse_scratch_doubles(M->coarse_sys) > NOALLOC_COARSE_DOUBLES)
    return fail(M, HHG_EINVAL,
                "coarsest level needs " + std::to_string(coarse_scratch_doubles(M->coarse_sys)) +
                    " scratch doubles; the allocation-free coarse solve holds " +
                    std::to_string(NOALLOC_COARSE_DOUBLES));
  CK(cudaSetDevice(M->device));
  LevelHost& H = M->lv[M->coarsest];
  LevelDev<double>& L = H.d64;
  const int64_t n = H.sh.n();
  int rc;
  // inputs into the coarsest-level fields through the mesh's staging buffer
  if ((rc = stage_in(M, f, 3 * n))) return rc;
  launch_scatter(L, M->d_stage, 3, L.f, F_VFREE, M->stream);
  if ((rc = stage_in(M, u, 3 * n))) return rc;
  launch_scatter(L, M->d_stage, 3, L.u, F_VFREE, M->stream);
  double* gp[1] = {L.g};
  if ((rc = stage_in(M, g, n))) return rc;
  launch_scatter(L, M->d_stage, 1, gp, F_ACT, M->stream);
  double* pp[1] = {L.p};
  if ((rc = stage_in(M, p, n))) return rc;
  launch_scatter(L, M->d_stage, 1, pp, F_ACT, M->stream);
  CoarseParams prm{M->opt.coarse_minres_max, M->opt.coarse_minres_rtol, M->opt.coarse_cg_max, M->opt.coarse_cg_rtol};
  if ((rc = coarse_solve_noalloc(M->coarse_sys, L, prm, M->d_scalars + 5, M->stream, M->err))) return rc;
  M->launches += 5;
  const double* us[3] = {L.u[0], L.u[1], L.u[2]};
  launch_gather<double>(L, us, 3, M->d_stage, M->stream);
  if ((rc = stage_out(M, u, 3 * n))) return rc;
  const double* ps[1] = {L.p};
  launch_gather<double>(L, ps, 1, M->d_stage, M->stream);
  if ((rc = stage_out(M, p, n))) return rc;
  M->launches += 2;
  CK(cudaGetLastError());
  return HHG_OK;
}

int hhg_level_op(hhg_mesh* M, int32_t level, int32_t precision, int32_t op, int32_t count) {
  int rc = check_level(M, level);
  if (rc) return rc;
  if ((precision != 0 && precision != 1) || count < 0) return fail(M, HHG_EINVAL, "bad precision or count");
  CK(cudaSetDevice(M->device));
  if (precision == 1 && (rc = ensure32(M))) return rc;
  // fixed-point refinement: Q from the FP64 iterate first, checked after
  // every step, and the FP64 iterate written back at the end
  const bool fx = precision == 1 && M->opt.ir_fixed_point && (op == HHG_OP_REFINE || op == HHG_OP_CYCLE) &&
                  level == M->finest && count > 0;
  if (fx) enq_ir_residual(M, false);
  for (int it = 0; it < count; ++it) {
    if ((rc = enqueue_op(M, level, precision, op))) return rc;
    CK(cudaGetLastError());
    if (fx) {
      CK(cudaMemcpyAsync(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost, M->stream));
      CK(cudaStreamSynchronize(M->stream));
      if ((rc = fx_recover_if_flagged(M))) return rc;
    }
  }
  if (fx) fx_materialize(M);
  CK(cudaMemcpyAsync(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return tile_status(M);
}

int hhg_time_op(hhg_mesh* M, int32_t level, int32_t precision, int32_t op, int32_t reps, double* ms) {
  int rc = check_level(M, level);
  if (rc) return rc;
  if ((precision != 0 && precision != 1) || reps < 1 || !ms) return fail(M, HHG_EINVAL, "bad arguments");
  CK(cudaSetDevice(M->device));
  if (precision == 1 && (rc = ensure32(M))) return rc;
  const bool fx = precision == 1 && M->opt.ir_fixed_point && (op == HHG_OP_REFINE || op == HHG_OP_CYCLE) &&
                  level == M->finest;
  if (fx) enq_ir_residual(M, false);
  if ((rc = enqueue_op(M, level, precision, op))) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaStreamSynchronize(M->stream));
  cudaEventRecord(e0, M->stream);
  for (int it = 0; it < reps && rc == 0; ++it) rc = enqueue_op(M, level, precision, op);
  cudaEventRecord(e1, M->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(M, e, "time_op");
  *ms = (double)t / reps;
  if (fx) fx_materialize(M);
  CK(cudaMemcpy(M->h_scalars, M->d_scalars, sizeof(double) * 16, cudaMemcpyDeviceToHost));
  return tile_status(M);
}

int hhg_kernel_launches(const hhg_mesh* mesh, int64_t* count) {
  if (!mesh || !count) return HHG_EINVAL;
  *count = mesh->launches;
  return HHG_OK;
}

int hhg_allocations(const hhg_mesh* mesh, int64_t* count) {
  if (!mesh || !count) return HHG_EINVAL;
  *count = mesh->allocations;
  return HHG_OK;
}

static int enqueue_op(hhg_mesh* M, int32_t level, int32_t precision, int32_t op) {
  {
    switch (op) {
      case HHG_OP_UZAWA_STEP:
        precision ? enq_uzawa<float>(M, level) : enq_uzawa<double>(M, level);
        break;
      case HHG_OP_VEL_FORWARD:
        precision ? enq_vel_sweep<float>(M, level, true) : enq_vel_sweep<double>(M, level, true);
        break;
      case HHG_OP_VEL_BACKWARD:
        precision ? enq_vel_sweep<float>(M, level, false) : enq_vel_sweep<double>(M, level, false);
        break;
      case HHG_OP_VEL_RHS:
        precision ? launch_vel_rhs<float>(M->lv[level].d32, M->stream) : launch_vel_rhs<double>(M->lv[level].d64, M->stream);
        break;
      case HHG_OP_PRES_RHS:
        precision ? launch_pres_rhs<float>(M->lv[level].d32, M->stream) : launch_pres_rhs<double>(M->lv[level].d64, M->stream);
        break;
      case HHG_OP_PRES_SWEEP:
        precision ? enq_pres_sweep<float>(M, level) : enq_pres_sweep<double>(M, level);
        break;
      case HHG_OP_RESIDUAL:
        precision ? launch_residual<float>(M->lv[level].d32, M->stream) : launch_residual<double>(M->lv[level].d64, M->stream);
        break;
      case HHG_OP_RESTRICT:
        if (level == M->coarsest) return fail(M, HHG_EINVAL, "no coarser level");
        precision ? launch_restrict<float>(M->lv[level].d32, M->lv[level - 1].d32, M->stream)
                  : launch_restrict<double>(M->lv[level].d64, M->lv[level - 1].d64, M->stream);
        break;
      case HHG_OP_PROLONG_ADD:
        if (level == M->coarsest) return fail(M, HHG_EINVAL, "no coarser level");
        precision ? launch_prolong_add<float>(M->lv[level].d32, M->lv[level - 1].d32, M->stream)
                  : launch_prolong_add<double>(M->lv[level].d64, M->lv[level - 1].d64, M->stream);
        break;
      case HHG_OP_COARSE_SOLVE:
        if (level != M->coarsest) return fail(M, HHG_EINVAL, "coarse solve runs on the coarsest level");
        precision ? enq_coarse<float>(M) : enq_coarse<double>(M);
        break;
      case HHG_OP_VCYCLE:
        precision ? enq_vcycle<float>(M, level) : enq_vcycle<double>(M, level);
        break;
      case HHG_OP_VEL_FORWARD_F:
        precision ? enq_vel_sweep_f<float>(M, level) : enq_vel_sweep_f<double>(M, level);
        break;
      case HHG_OP_PRES_SWEEP_F:
        precision ? enq_pres_sweep_f<float>(M, level) : enq_pres_sweep_f<double>(M, level);
        break;
      case HHG_OP_PROJECT:
        precision ? enq_project<float>(M, level) : enq_project<double>(M, level);
        break;
      case HHG_OP_REFINE:
        if (level != M->finest || !precision) return fail(M, HHG_EINVAL, "refinement runs on the finest level in FP32");
        if (M->opt.ir_fixed_point)
          launch_fx_update(M->fx, M->lv[level].d32, fx_state(M), M->lv[level].nalloc, M->stream);
        else
          launch_ir_update(M->lv[level].d64, M->lv[level].d32, M->stream);
        M->launches += 1;
        enq_slip_fix(M, level, M->opt.ir_fixed_point != 0);
        enq_ir_residual(M, M->opt.ir_fixed_point != 0);
        break;
      case HHG_OP_CYCLE:
        if (level != M->finest) return fail(M, HHG_EINVAL, "a solver cycle is rooted at the finest level");
        precision ? enq_cycle32(M) : enq_cycle64(M);
        break;
      case HHG_OP_FUSED_PASS0:
      case HHG_OP_FUSED_PASS1:
      case HHG_OP_FUSED_PASS2:
        if (!precision || !M->lv[level].fused) return fail(M, HHG_EINVAL, "the level has no fused FP32 passes");
        enq_uzawa_fused(M, level, op - HHG_OP_FUSED_PASS0);
        break;
      default:
        return fail(M, HHG_EINVAL, "unknown op");
    }
  }
  return HHG_OK;
}

}  // extern "C"
