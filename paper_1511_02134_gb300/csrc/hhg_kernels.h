// Host-side launchers of the level kernels (hhg_kernels.cu, hhg_coarse.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hhg_device.cuh"

namespace hhg {

// Smoother pieces (Sec. 3.3 inexact Uzawa step, Sec. 3.5 smoothers)
template <class T> void launch_vel_rhs(const LevelDev<T>& L, cudaStream_t s);
template <class T> void launch_vel_colour(const LevelDev<T>& L, int colour, cudaStream_t s);
template <class T> void launch_pres_rhs(const LevelDev<T>& L, cudaStream_t s);
template <class T> void launch_pres_colour(const LevelDev<T>& L, int colour, cudaStream_t s);
// Colour sweeps that form their right-hand side at each node (f - B^T p for
// velocity, B u - g for pressure) instead of reading RU / RP.
template <class T> void launch_vel_colour_rhs(const LevelDev<T>& L, int colour, cudaStream_t s);
template <class T> void launch_pres_colour_rhs(const LevelDev<T>& L, int colour, cudaStream_t s);
// Backward velocity colour 0 and pressure colour 0 in one launch (the
// velocity right-hand side read from RU when ru, else formed at the node).
template <class T> void launch_vel_pres_colour0(const LevelDev<T>& L, bool ru, cudaStream_t s);
// Colour-fused FP32 Uzawa step (hhg_fused.cu): three passes over a level,
// each a z-march of CTAs over (x, y) tiles with F colour phases per march
// step on planes staged into a shared-memory ring by tensor copies:
//   kind 0: velocity colours 0 1 2 3, (U, P) -> RU;
//   kind 1: velocity colours 2 1, then velocity + pressure colour 0,
//           (RU, P) -> (U, RP);
//   kind 2: pressure colours 1 2 3, (U, RP) -> P.
// TileMaps holds the tensor maps of the four staged input fields of one pass.
// A CTA whose bounded wait for a copy runs out writes HHG_TILE_TIMEOUT to
// *err and stops after its copies have landed (HHG_TILE_DRAIN_TIMEOUT if
// even that bounded wait runs out).
struct TileMaps {
  CUtensorMap m[4];
};
constexpr unsigned HHG_TILE_TIMEOUT = 0x7117u;
constexpr unsigned HHG_TILE_DRAIN_TIMEOUT = 0x7118u;
constexpr int FUSED_MAX_THREADS = 640;
constexpr long long FUSED_WAIT_POLLS = 1ll << 20;  // default bound of one mbarrier wait
// Default of hhg_options.fused_min_nodes: never.  Measured on GB300 (cube,
// FP32 Uzawa step): level 9 12.0 ms fused against 6.8 ms with the colour
// launches, level 8 2.4 against 1.0 ms.  The passes move 1.1x their
// algorithmic DRAM bytes but are bound on the SM side: one CTA per SM (its
// plane ring fills the shared memory), a few hundred node updates per colour
// phase between barriers, about 30 shared-memory loads per update.
constexpr int64_t FUSED_MIN_NODES = -1;
struct FusedArgs {
  int by, ty;      // staged rows (ty + 2 F) and the tile's rows
  int fstride;     // floats between staged fields in shared memory
  long long polls; // bound of one mbarrier wait
  int extra_tx;    // tests: bytes announced beyond what the first staged plane delivers
  unsigned* err;   // error word
  float* out_u[3]; // output velocity (kinds 0, 1)
  float* out_p;    // output pressure (kinds 1, 2)
};
struct FusedPlan {
  int ntx;                          // tiles in x (64 nodes each, the first 67)
  int ty[3], by[3], nty[3];         // per kind: tile rows, staged rows, tiles in y
  TileMaps maps[3];                 // per kind: maps of its input fields
};
int fused_tiles_x(int nx);
// Tile heights (ty_override > 0 forces one) and tensor maps of a level's FP32
// fields; call after the FP32 fields are allocated.
int plan_fused(const LevelDev<float>& L, int ty_override, FusedPlan& P, std::string& err);
void launch_uzawa_pass(const FusedPlan& P, const LevelDev<float>& L, int kind, unsigned* err, long long polls,
                       int extra_tx, cudaStream_t s);
// Shared-memory limits of the pass kernels (once per device).
void prepare_fused();
// Default of hhg_options.spec_max_nodes: levels below 2^20 lattice nodes are
// latency bound and use the speculative node form of the colour updates
// (hhg_node_ops.cuh).  Measured on GB300: a level-5 FP32 Uzawa step 37.9 ->
// 28.2 us, level 6 60 -> 49 us, while level 7 went 170 -> 191 us.
constexpr int64_t SPEC_MAX_NODES = 1 << 20;
// Residual (RU, RP) = (F, G) - K (U, P); zero on nodes without unknowns.
template <class T> void launch_residual(const LevelDev<T>& L, cudaStream_t s);

// Transfers between level l (fine) and l-1 (coarse).
template <class T> void launch_restrict(const LevelDev<T>& fine, const LevelDev<T>& coarse, cudaStream_t s);
template <class T> void launch_prolong_add(const LevelDev<T>& fine, const LevelDev<T>& coarse, cudaStream_t s);

// Reductions: partial sums per block (REDUCE_BLOCKS of them, `width` values
// each) followed by a fixed-order final sum into out[0..width).
constexpr int REDUCE_BLOCKS = 304;
constexpr int REDUCE_THREADS = 256;
template <class T> void launch_residual_norm2(const LevelDev<T>& L, double* partial, double* out, cudaStream_t s);
template <class T> void launch_mass_moments(const LevelDev<T>& L, double* partial, double* out, cudaStream_t s);
// P -= moments[0] / moments[1] on active nodes.
template <class T> void launch_project(const LevelDev<T>& L, const double* moments, cudaStream_t s);

// Zero every field of the set {U, P} (what = 0), {F, G} (1), {RU, RP} (2).
template <class T> void launch_zero(const LevelDev<T>& L, int what, cudaStream_t s);

// Right-hand side of the finest level from staged nodal arrays (padded
// layout, component planes): fnod[3], uD[3] (uD zero off Dirichlet nodes).
// The arrays are quantized in place to int64 (one power-of-two scale for f,
// one for u_D, from their max |v| into mx[0..8) and sh[0..2)) and the
// regular-node stencils summed exactly in integers; the boundary nodes (irr,
// lattice coordinates as FxState::irr) use their class rows in FP64.
void launch_set_rhs(const LevelDev<double>& L, double* const* fnod, double* const* uD, unsigned long long* mx,
                    int* sh, const int64_t* irr, int64_t nirr, cudaStream_t s);
// D form: the Dirichlet lift of launch_set_rhs (its staged, quantized u_D
// and shifts) used A_1 per component; this adds A_1 u_D and subtracts
// A_2 u_D on the velocity nodes.
void launch_lift_d(const LevelDev<double>& L, double* const* uD, const int* sh, cudaStream_t s);
// G -= mean(G) over active nodes (two passes through partial/out).
void launch_remove_mean_g(const LevelDev<double>& L, double* partial, double* out, cudaStream_t s);

// Gradient of the right-hand side map: grad_f[d] = M lam_u[d] + G_d^T lam_p
// with lam fields in L.u / L.p of an FP64 level, written to out[3] (padded).
void launch_rhs_transpose(const LevelDev<double>& L, double* const* out, cudaStream_t s);

// Mixed precision: FP64 residual of (x, b) written as FP32 into e.f/e.g,
// squared norm partials; and x += e.
void launch_ir_residual(const LevelDev<double>& x, const LevelDev<float>& e, double* partial, double* out,
                        cudaStream_t s);
// x += e in FP64.
void launch_ir_update(const LevelDev<double>& x, const LevelDev<float>& e, cudaStream_t s);
// Fixed-point iterate of the FP32+IR solve (hhg_kernels.cu): per field
// Q = x 2^s with an integer per-field shift s, |Q| < 2^55, so that the
// regular-node stencils of the FP64 residual are exact 64-bit sums.  The
// cycle updates Q itself (launch_fx_update, no FP64 arithmetic); the FP64
// iterate x is written from Q at the end of a solve, or rebuilt as
// old iterate + e in FP64 when a check of the update fails (a correction too
// large for the shift, |Q| grown to 2^55 or shrunk below 2^45): the host then
// requantizes x with fresh shifts.  IR_BLOCKS blocks: the partial-sum buffer
// holds that many per value.
constexpr int IR_BLOCKS = 1216;
struct FxIterate {
  int64_t* u[3];
  int64_t* p;
};
struct FxState {
  unsigned long long* mx;    // [4] per-field max |x| (FP64 bits), quantization
  unsigned long long* maxq;  // [4] per-field max |Q| after an update
  int* exp;                  // [4] shifts s
  unsigned* flag;            // FX_FLAG_* bits, cleared by the host
  const int64_t* irr;        // lattice coordinates (k << 42) | (j << 21) | i of the F_IRR nodes
  int64_t nirr;
};
// Blocks of the boundary-node part of the fixed-point residual (its partial
// sums follow the IR_BLOCKS of the regular part).
constexpr int IR_IRR_BLOCKS = 304;
constexpr unsigned FX_FLAG_REFUSED = 1u;  // k_fx_update left a correction out
constexpr unsigned FX_FLAG_RESCALE = 2u;  // the residual found the iterate unfit for its shifts
// Residual of the fixed-point iterate into e.f / e.g, norm into out[0].
// from_update = false: max |x| -> shifts -> Q = round(x 2^s) first;
// true: Q comes from launch_fx_update and is checked first.  partial holds
// ir_residual_fx_partials(x) doubles (one per block of the regular-node
// kernel, then the boundary-node blocks and the segment sums).
void launch_ir_residual_fx(const LevelDev<double>& x, const FxIterate& q, const LevelDev<float>& e, const FxState& st,
                           bool from_update, double* partial, double* out, cudaStream_t s);
// Free slip: the velocity of the slip nodes among the listed boundary nodes
// (irr: lattice coordinates as in FxState::irr) made tangential in FP64, on
// the FP64 iterate or on the fixed-point one (FX_FLAG_RESCALE if a value
// leaves the checked range).
void launch_slip_fix(const LevelDev<double>& x, const int64_t* irr, int64_t nirr, cudaStream_t s);
void launch_slip_fix_fx(const FxIterate& q, const LevelDev<double>& x, const FxState& st, cudaStream_t s);
// Q += round(e 2^s) over the nalloc padded positions.
int64_t ir_residual_fx_partials(const LevelDev<double>& x);
void launch_fx_update(const FxIterate& q, const LevelDev<float>& e, const FxState& st, int64_t nalloc, cudaStream_t s);
// x = Q 2^-s, or (recover) the iterate before the last update + e in FP64.
void launch_fx_to_fp64(const LevelDev<double>& x, const FxIterate& q, const LevelDev<float>& e, const FxState& st,
                       bool recover, cudaStream_t s);

// Layout conversion between contiguous (n, 3)/(n,) arrays and padded fields.
// mask: nodes whose value is kept (others get 0); 0 = keep all.
void launch_scatter(const LevelDev<double>& L, const double* src, int ncomp, double* const* dst, uint8_t mask,
                    cudaStream_t s);
template <class T>
void launch_gather(const LevelDev<T>& L, const T* const* src, int ncomp, double* dst, cudaStream_t s);
// u_out[dir] = values of the compact Dirichlet list
void launch_dirichlet_fill(const int64_t* idx, const double* val, int64_t ndir, const LevelDev<double>& L, double* dst,
                           cudaStream_t s);
// val (3 per entry) = U at the padded indices pad (compact Dirichlet data)
void launch_dirichlet_gather(const int64_t* pad, int64_t ndir, const LevelDev<double>& L, double* val,
                             cudaStream_t s);
void launch_cast_field(const double* src, float* dst, int64_t n, cudaStream_t s);
// Coarse level's RU (body force, active nodes) and U (Dirichlet data,
// Dirichlet nodes) from the finest level's, node (i, j, k) taken from
// (stride i, stride j, stride k) of the finest.
void launch_inject(const LevelDev<double>& fine, const LevelDev<double>& coarse, int stride, cudaStream_t s);
// U at the listed padded indices = val (3 per entry): the inverse of launch_dirichlet_gather.
void launch_dirichlet_scatter(const int64_t* pad, int64_t ndir, const double* val, const LevelDev<double>& L,
                              cudaStream_t s);
void launch_scale(double* x, int64_t n, double a, cudaStream_t s);

// Coarse-grid solver (hhg_coarse.cu): (U, P) += PMINRES correction of the
// residual equation, FP64 on the compact unknowns of the coarsest level.
// CoarseSys is the device view of the assembled CoarseMatrix (hhg_lattice.h).
struct CoarseSys {
  int32_t nv, np;         // velocity unknowns per component, pressure unknowns
  int32_t coupled;        // D form: A is the coupled 3 nv x 3 nv velocity block
  const int32_t* vidx;    // padded lattice index of each velocity unknown's node
  const int32_t* pidx;    // padded lattice index of each pressure unknown's node
  const int32_t* kptr;    // K in CSR, 3 nv + np rows
  const int32_t* kcol;
  const double* kval;
  const int32_t* aptr;    // scalar A in CSR, nv rows
  const int32_t* acol;
  const double* aval;
  const double* mass;     // lumped mass of each pressure unknown
};
struct CoarseParams {
  int minres_max;
  double minres_rtol;
  int cg_max;
  double cg_rtol;
};
// Scratch doubles of one coarse solve: 11 vectors of 3 nv + np entries and 9 nv.
__host__ __device__ inline int64_t coarse_scratch_doubles(const CoarseSys& S) {
  return 11 * (3 * (int64_t)S.nv + S.np) + 9 * (int64_t)S.nv;
}
// A coarsest level this small is solved by one thread block (one warp per CG).
constexpr int64_t COARSE_BLOCK_MAX_UNKNOWNS = 4096;
__host__ __device__ inline bool coarse_fits_block(const CoarseSys& S) {
  return 3 * (int64_t)S.nv + S.np <= COARSE_BLOCK_MAX_UNKNOWNS;
}
template <class T>
void launch_coarse_solve(const CoarseSys& S, const LevelDev<T>& L, double* scratch, CoarseParams prm, double* info,
                         cudaStream_t s);
// Cluster set-up of the coarse solve (call once per device before launches).
void prepare_coarse_solve();

// Same solve with its scratch in a file-scope device array (no allocation).
// Fails with HHG_EINVAL when coarse_scratch_doubles(S) exceeds the array.
constexpr int64_t NOALLOC_COARSE_DOUBLES = 1 << 18;
constexpr int NOALLOC_MAX_DEVICES = 64;
int coarse_solve_noalloc(const CoarseSys& S, const LevelDev<double>& L, CoarseParams prm, double* info,
                         cudaStream_t s, std::string& err);

// Fused cycle of the coarse levels (hhg_small.cu): levels lv[0] (coarsest)
// .. lv[nlev-1] of one hierarchy run by one cluster of nblocks CTAs,
// smoothing counts per level, the compact system of the coarsest level for
// the coarse solve, its scratch and parameters.
constexpr int SMALL_MAX_LEVELS = 8;
// Defaults, measured on GB300 with whole level-7 cube solves: fusing only the
// levels of at most 1024 nodes into one block is fastest in both precisions.
// Larger fused levels lose to the per-level kernels (FP64: one SM has 1/152
// of the FP64 rate), and cluster-wide fusion, although its V-cycles are fast
// in isolation, slows the solve down between the other kernels of a cycle.
constexpr int64_t SMALL_MAX_NODES = 1024;
constexpr int64_t SMALL_MAX_NODES_FP64 = 1024;
constexpr unsigned SMALL_TEAM_BLOCKS = 1;
constexpr unsigned SMALL_TEAM_BLOCKS_FP64 = 1;
template <class T>
struct SmallCycle {
  unsigned nblocks;
  LevelDev<T> lv[SMALL_MAX_LEVELS];
  int nlev;
  int nu_pre[SMALL_MAX_LEVELS];
  int nu_post[SMALL_MAX_LEVELS];
  T inv6nuh[SMALL_MAX_LEVELS];
  T omc[SMALL_MAX_LEVELS];
  CoarseSys cs;
  double* scratch;
  CoarseParams prm;
  double* info;
};
template <class T>
void launch_small_cycle(const SmallCycle<T>& S, cudaStream_t s);
// Cluster-resident cycle of the coarse levels (hhg_resident.cu): levels
// lv[1..nres] live in the shared memory of one thread-block cluster of
// nblocks CTAs, split into runs of z-planes over the first nbq[q] CTAs (CTA r
// holds node planes [kb[q][r], kb[q][r+1]) of level q, kb[q][r] =
// ceil(r nz / nbq[q])), and are
// read across CTAs through distributed shared memory; lv[0], the coarsest
// level, stays in global memory for the coarse solve.  The kernel runs the
// part of the V_var cycle from lv[nres] (whose u, p, f, g it reads from and
// whose u, p it writes back to global memory) down to the coarse solve and
// back up.  Each CTA's dynamic shared memory holds, at the byte offsets
// below, a table of plane pointers per level (RES_TAB_FIELDS rows of pz
// generic pointers), a copy of its class-row table, one zero plane and a
// block per level: RES_FIELDS fields
// of type T (u_0, u_1, u_2, p, f_0, f_1, f_2, g), then the node flags (bytes)
// and stencil classes (16 bit), each maxpl[q] padded planes.
constexpr int RES_MAX_LEVELS = 4;
constexpr int64_t RES_MAX_NODES = 1 << 16;  // default cap on the top level's lattice nodes
// Default cluster sizes, from whole level-7 cube solves on GB300 (FP32+IR
// 38.4 -> 37.3 ms with 8 CTAs, FP64 112.5 -> 109.5 ms with 16; both hold
// levels 3 and 4, level 5 does not fit).  Each colour phase still costs
// about 2.5 us: the chain of dependent loads of a boundary node (flags,
// class, weights, neighbours) sets it, whether the phase is a launch, a
// phase of the global-memory fused kernel or a phase here.
constexpr unsigned RES_CTAS_FP32 = 8;
constexpr unsigned RES_CTAS_FP64 = 16;
constexpr int RES_MAX_CTAS = 16;
constexpr int RES_LISTS = 16;
constexpr int RES_FIELDS = 12;
constexpr int RES_TAB_FIELDS = 14;
template <class T>
struct ResidentCycle {
  unsigned nblocks;
  int nres;
  LevelDev<T> lv[RES_MAX_LEVELS + 1];
  int nu_pre[RES_MAX_LEVELS + 1];
  int nu_post[RES_MAX_LEVELS + 1];
  T inv6nuh[RES_MAX_LEVELS + 1];
  T omc[RES_MAX_LEVELS + 1];
  int nbq[RES_MAX_LEVELS + 1];  // CTAs holding level q (the first nbq[q] of the cluster)
  int kb[RES_MAX_LEVELS + 1][RES_MAX_CTAS + 1];
  int maxpl[RES_MAX_LEVELS + 1];
  int ncls[RES_MAX_LEVELS + 1];  // boundary stencil classes of the level (table rows 0..ncls)
  uint32_t tab[RES_MAX_LEVELS + 1];
  uint32_t wts[RES_MAX_LEVELS + 1];  // byte offset of the level's class table copy
  uint32_t blk[RES_MAX_LEVELS + 1];
  uint32_t zero;
  uint32_t smem;
  // Node lists of level q (RES_LISTS of them, list l = 8 kind + 2 colour +
  // boundary, with kind 0 velocity (F_VFREE) / 1 pressure (F_ACT) and
  // boundary 0 regular / 1 F_IRR): entries (k << 20) | (j << 10) | i in
  // lattice order (sorted by k), list l at lists[q][loff[q][l] .. loff[q][l + 1]).
  // (null: the level's colour phases test flags at every lattice position).
  const int32_t* lists[RES_MAX_LEVELS + 1];
  int32_t loff[RES_MAX_LEVELS + 1][RES_LISTS + 1];
  uint32_t lst[RES_MAX_LEVELS + 1];  // byte offset of the CTA's copy of its part of the lists
  uint32_t lofs;  // byte offset of the per-level offsets of that copy and of its sources
  CoarseSys cs;
  double* scratch;
  CoarseParams prm;
  double* info;
};
// Plans the shared-memory layout of levels lv[1..nres]: the CTAs per level
// (nbq, at most max_ctas; nblocks = the largest), kb, maxpl, and the offsets;
// false if it cannot fit smem_limit bytes per CTA.
template <class T>
bool plan_resident(ResidentCycle<T>& S, size_t smem_limit, unsigned max_ctas);
template <class T>
cudaError_t launch_resident_cycle(const ResidentCycle<T>& S, cudaStream_t s);
// Cluster size (16, else 8) and the dynamic shared memory available to one
// CTA of the resident kernel; sets the kernel attributes.
template <class T>
unsigned prepare_resident(size_t& smem_limit);
// Cluster size for the fused cycle (16, else 8); sets kernel attributes.
unsigned prepare_small_cycle();

}  // namespace hhg
