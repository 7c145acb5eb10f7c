// Level kernels of the all-at-once Uzawa multigrid (Sec. 3.3-3.6).
//
// Every kernel works on one level of the padded lattice (hhg_device.cuh).
// Colour kernels update the nodes with (i + j + k) mod 4 == colour; these
// are not coupled by the 15-point pattern of the operator, so one launch per
// colour performs the Gauss-Seidel sweep in colour order.
#include <type_traits>

#include "hhg_kernels.h"
#include "hhg_node_ops.cuh"

namespace hhg {

namespace {

constexpr int CB = 128;  // colour kernels: packed (row, quarter-row slot) indices per block; planes per level (cbz)
// (blocks of CB x cbz threads, cbz <= 4: the colour kernels are compiled for 4 CB threads per block)
constexpr int FX = 64, FY = 4;  // full kernels
constexpr int IR_FZ = 8;        // planes per block of the fixed-point residual

template <class T>
dim3 colour_block(const LevelDev<T>& L) {
  return dim3(CB, 1, L.cbz);
}
template <class T>
dim3 colour_grid(const LevelDev<T>& L) {
  const int64_t slots = (int64_t)L.ny * L.nq;
  return dim3((unsigned)((slots + CB - 1) / CB), (unsigned)((L.nz + L.cbz - 1) / L.cbz), 1);
}
template <class T>
dim3 full_grid(const LevelDev<T>& L) {
  return dim3((L.nx + FX - 1) / FX, (L.ny + FY - 1) / FY, L.nz);
}

// Whether the level's colour kernels use the speculative node form
// (hhg_node_ops.cuh); set per level by the host (hhg_options.spec_max_nodes).
template <class T>
bool spec_level(const LevelDev<T>& L) {
  return L.spec != 0;
}

// Colour-kernel node: returns false if outside the lattice.
template <class T>
__device__ __forceinline__ bool colour_node(const LevelDev<T>& L, int colour, int& i, int& j, int& k) {
  // slot t of plane k: row j = t / nq, quarter-row slot t - j nq (the rows of
  // a plane packed back to back, so that no warp holds only a row's tail)
  const uint64_t t = (uint64_t)blockIdx.x * CB + threadIdx.x;
  k = blockIdx.y * blockDim.z + threadIdx.z;
  const uint64_t row = L.nq == 1 ? t : __umul64hi(t, L.nq_mul);
  if (row >= (uint64_t)L.ny) return false;
  j = (int)row;
  i = ((colour - j - k) & 3) + 4 * (int)(t - row * (uint64_t)L.nq);
  return i < L.nx && k < L.nz;
}

template <class T>
__device__ __forceinline__ bool full_node(const LevelDev<T>& L, int& i, int& j, int& k) {
  i = blockIdx.x * FX + threadIdx.x;
  j = blockIdx.y * FY + threadIdx.y;
  k = blockIdx.z;
  return i < L.nx && j < L.ny;
}

// ---- smoother, residual, transfers: grid kernels over the per-node bodies ----------

// RU = F - B^T P on velocity nodes (the right-hand side of both velocity
// sweeps of one Uzawa step, Sec. 3.3).
template <class T>
__global__ void k_vel_rhs(LevelDev<T> L) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  node_vel_rhs(L, node_at(L.px, L.pxy, i, j, k));
}

// Gauss-Seidel update of the velocity nodes of one colour.  SPEC: the
// speculative node form of small levels (hhg_node_ops.cuh).
// DF: the velocity block's form (1 D form, 0 Laplace form; hhg_node_ops.cuh).
template <class T, bool SPEC, int DF>
__global__ void __launch_bounds__(CB * 4) k_vel_colour(LevelDev<T> L, int colour, T inv6nuh) {
  pdl_enter();
  int i, j, k;
  if (!colour_node(L, colour, i, j, k)) return;
  node_vel_gs<SPEC, T, DF>(L, node_at(L.px, L.pxy, i, j, k), inv6nuh);
}

template <class T, bool SPEC, int DF>
__global__ void __launch_bounds__(CB * 4) k_vel_colour_rhs(LevelDev<T> L, int colour, T inv6nuh) {
  pdl_enter();
  int i, j, k;
  if (!colour_node(L, colour, i, j, k)) return;
  node_vel_gs_rhs<SPEC, T, DF>(L, node_at(L.px, L.pxy, i, j, k), inv6nuh);
}

// The last velocity colour of a step (backward colour 0) and the first
// pressure colour in one launch.  A pressure node of colour 0 reads the
// velocity of its neighbours, which are of the other colours and final
// after the earlier colour launches, and its own velocity, which the same
// thread has just updated; the velocity update reads the old pressure of
// the node and of its neighbours, none of which this launch changes before
// the node's own pressure update.  So the sequential order is kept.
// RU: the velocity right-hand side is read from RU (FP64 path) instead of
// being formed at the node.
template <class T, bool RU, bool SPEC, int DF>
__global__ void __launch_bounds__(CB * 4) k_vel_pres_colour0(LevelDev<T> L, T inv6nuh, T omega_over_6c) {
  pdl_enter();
  int i, j, k;
  if (!colour_node(L, 0, i, j, k)) return;
  const Node n = node_at(L.px, L.pxy, i, j, k);
  if (RU)
    node_vel_gs<SPEC, T, DF>(L, n, inv6nuh);
  else
    node_vel_gs_rhs<SPEC, T, DF>(L, n, inv6nuh);
  node_pres_gs_rhs<SPEC>(L, n, omega_over_6c);
}

template <class T, bool SPEC>
__global__ void __launch_bounds__(CB * 4) k_pres_colour_rhs(LevelDev<T> L, int colour, T omega_over_6c) {
  pdl_enter();
  int i, j, k;
  if (!colour_node(L, colour, i, j, k)) return;
  node_pres_gs_rhs<SPEC>(L, node_at(L.px, L.pxy, i, j, k), omega_over_6c);
}

// ---- FP32 colour kernels with two nodes per thread -------------------------------
// On rows grouped by x mod 4, the nodes of one colour sit at consecutive
// positions of one residue group.  A thread takes the two nodes at positions
// 2p, 2p + 1 (8-byte aligned: row pitches are multiples of 16 entries), and
// every neighbour pair it reads lies at two consecutive positions too; the
// pairs of its y and z neighbours and of its x neighbours in the adjacent
// residue groups are aligned, except the x - 1 pair of residue 0 and the
// x + 1 pair of residue 3, read as two values.  Where both nodes take the
// closed-form update (regular, with the unknown), the thread evaluates the
// per-node expressions of hhg_node_ops.cuh on the pair (half the load
// instructions, twice the bytes per load); otherwise each node runs the
// per-node body.

struct F2 {
  float x, y;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ F2(float s) : x(s), y(s) {}
  __device__ __forceinline__ F2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(a.x * b.x, a.y * b.y); }

// Pair view centred on the node pair at entry c (first node).
struct PairNb {
  const float* x;
  int64_t c, dxm, dxp, px, pxy;
  bool am, ap;  // the x - 1 / x + 1 pair is 8-byte aligned
  __device__ __forceinline__ F2 operator()(int dx, int dy, int dz) const {
    const int64_t e = c + (dx < 0 ? dxm : (dx > 0 ? dxp : 0)) + px * dy + pxy * dz;
    if ((dx < 0 && !am) || (dx > 0 && !ap)) return F2(x[e], x[e + 1]);
    const float2 v = *reinterpret_cast<const float2*>(x + e);
    return F2(v.x, v.y);
  }
};

__device__ __forceinline__ F2 load2(const float* x, int64_t c) {
  const float2 v = *reinterpret_cast<const float2*>(x + c);
  return F2(v.x, v.y);
}
__device__ __forceinline__ void store2(float* x, int64_t c, F2 v) {
  *reinterpret_cast<float2*>(x + c) = make_float2(v.x, v.y);
}

// KIND 0: velocity colour with f - B^T p formed at the node; 1: pressure
// colour with B u - g formed at the node; 2: velocity colour 0 then pressure
// colour 0 (the last velocity and first pressure colour of a step).
template <int KIND>
__global__ void __launch_bounds__(CB * 4) k_colour_pair(LevelDev<float> L, int colour, float inv6nuh, float omc) {
  pdl_enter();
  const uint64_t t = (uint64_t)blockIdx.x * CB + threadIdx.x;
  const int k = blockIdx.y * blockDim.z + threadIdx.z;
  const uint64_t row = L.nq2 == 1 ? t : __umul64hi(t, L.nq2_mul);
  if (row >= (uint64_t)L.ny || k >= L.nz) return;
  const int j = (int)row;
  const int pp = (int)(t - row * (uint64_t)L.nq2);
  const int rho = (colour - j - k) & 3;             // i mod 4 of the colour's nodes in this row
  const int i0 = 4 * (2 * pp - ((rho + 1) >> 2)) + rho;  // at padded position 2 pp
  const int i1 = i0 + 4;
  const bool in0 = i0 >= 0 && i0 < L.nx, in1 = i1 < L.nx;
  if (!in0 && !in1) return;
  const int r = (rho + 1) & 3;                       // residue of padded x = i + 1
  const int64_t c0 = (int64_t)r * (L.px >> 2) + 2 * pp + L.px * (j + 1) + L.pxy * (k + 1);
  const uint8_t fl0 = in0 ? L.flags[c0] : (uint8_t)0, fl1 = in1 ? L.flags[c0 + 1] : (uint8_t)0;
  const uint8_t need = KIND == 1 ? F_ACT : (KIND == 2 ? (F_ACT | F_VFREE) : F_VFREE);
  const bool fast = ((fl0 & need) == need) && ((fl1 & need) == need) && !((fl0 | fl1) & F_IRR);
  if (!fast) {
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      const int i = q ? i1 : i0;
      if (!(q ? in1 : in0)) continue;
      const Node n = node_at(L.px, L.pxy, i, j, k);
      if (KIND == 0) node_vel_gs_rhs<false>(L, n, inv6nuh);
      if (KIND == 1) node_pres_gs_rhs<false>(L, n, omc);
      if (KIND == 2) {
        node_vel_gs_rhs<false>(L, n, inv6nuh);
        node_pres_gs_rhs<false>(L, n, omc);
      }
    }
    return;
  }
  const int64_t dxm = row_step_minus(i0 + 1, L.px), dxp = row_step_plus(i0 + 1, L.px);
  const bool am = r != 0, ap = r != 3;
  const PairNb u[3] = {PairNb{L.u[0], c0, dxm, dxp, L.px, L.pxy, am, ap},
                       PairNb{L.u[1], c0, dxm, dxp, L.px, L.pxy, am, ap},
                       PairNb{L.u[2], c0, dxm, dxp, L.px, L.pxy, am, ap}};
  const PairNb p{L.p, c0, dxm, dxp, L.px, L.pxy, am, ap};
  if (KIND != 1) {
    // the closed-form velocity update (vel_regular_value) on the pair
    F2 dv[3];
    div12_all(diff7v<F2>(p), dv);
    const F2 s = F2(-L.h2 * (1.0f / 12.0f));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const F2 v = ((load2(L.f[d], c0) - s * dv[d]) + F2(L.nuh) * nb6v(u[d])) * F2(inv6nuh);
      store2(L.u[d], c0, v);
    }
  }
  if (KIND != 0) {
    // the closed-form pressure update (pres_regular_value) on the pair; the
    // pair's own velocities are not among the neighbours read
    const F2 d0 = div12(diff7v<F2>(u[0]), 0);
    const F2 d1 = div12(diff7v<F2>(u[1]), 1);
    const F2 d2 = div12(diff7v<F2>(u[2]), 2);
    const F2 pc = load2(L.p, c0);
    const F2 rp = F2(L.h2 * (1.0f / 12.0f)) * ((d0 + d1) + d2) - load2(L.g, c0);
    const F2 cp = F2(L.c) * (F2(6.0f) * pc - nb6v(p));
    store2(L.p, c0, pc + F2(omc) * (rp - cp));
  }
}

template <class T>
dim3 pair_grid(const LevelDev<T>& L) {
  const int64_t slots = (int64_t)L.ny * L.nq2;
  return dim3((unsigned)((slots + CB - 1) / CB), (unsigned)((L.nz + L.cbz - 1) / L.cbz), 1);
}

// RP = B U - G on pressure nodes.
template <class T>
__global__ void k_pres_rhs(LevelDev<T> L) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  node_pres_rhs(L, node_at(L.px, L.pxy, i, j, k));
}

// Under-relaxed Gauss-Seidel on C for the pressure nodes of one colour.
template <class T>
__global__ void __launch_bounds__(CB * 4) k_pres_colour(LevelDev<T> L, int colour, T omega_over_6c) {
  pdl_enter();
  int i, j, k;
  if (!colour_node(L, colour, i, j, k)) return;
  node_pres_gs(L, node_at(L.px, L.pxy, i, j, k), omega_over_6c);
}

template <class T, int DF>
__global__ void k_residual(LevelDev<T> L) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  node_residual<T, DF>(L, node_at(L.px, L.pxy, i, j, k));
}

// The residual of the Laplace form on large levels, four nodes per thread:
// the nodes at padded x = 4 pos .. 4 pos + 3 of one row, which sit at the
// same position pos of the four residue groups (rows grouped by x mod 4).
// Their 15-point stencils share most neighbours: per field the quad reads 36
// values (6 in its own row, 5 in each of the rows y +- 1, z +- 1, (y, z) +-
// (1, 1)) instead of 4 x 15, so each thread issues about half the loads of the
// per-node kernel.  A quad with a node outside the lattice, without an
// unknown or on the boundary (F_IRR) takes the per-node body for each of its
// nodes.  The arithmetic is that of node_residual_v for regular nodes.
struct QuadRows {
  int64_t c;        // padded index of the quad's first node (padded x = 4 pos, residue 0)
  int64_t g;        // entries per residue group, px / 4
  int64_t py, pz;   // row steps +y, +z
};

// The 6 values of the quad's own row (padded x = 4 pos - 1 .. 4 pos + 4), the
// 5 of a row above (x = 4 pos .. 4 pos + 4) or below (x = 4 pos - 1 .. 4 pos + 3).
template <class T>
__device__ __forceinline__ void quad_row6(const T* x, const QuadRows& q, int64_t r, T v[6]) {
  const int64_t b = q.c + r;
  v[0] = x[b + 3 * q.g - 1];
  v[1] = x[b];
  v[2] = x[b + q.g];
  v[3] = x[b + 2 * q.g];
  v[4] = x[b + 3 * q.g];
  v[5] = x[b + 1];
}
template <class T>
__device__ __forceinline__ void quad_row_up(const T* x, const QuadRows& q, int64_t r, T v[5]) {
  const int64_t b = q.c + r;
  v[0] = x[b];
  v[1] = x[b + q.g];
  v[2] = x[b + 2 * q.g];
  v[3] = x[b + 3 * q.g];
  v[4] = x[b + 1];
}
template <class T>
__device__ __forceinline__ void quad_row_down(const T* x, const QuadRows& q, int64_t r, T v[5]) {
  const int64_t b = q.c + r;
  v[0] = x[b + 3 * q.g - 1];
  v[1] = x[b];
  v[2] = x[b + q.g];
  v[3] = x[b + 2 * q.g];
  v[4] = x[b + 3 * q.g];
}

// One field around the quad: centre, the six axis neighbours' sum and the
// seven antisymmetric differences of each of the four nodes.
template <class T>
struct QuadField {
  T ctr[4], nb6[4];
  Diff7<T> d[4];
};

template <class T>
__device__ __forceinline__ QuadField<T> quad_field(const T* x, const QuadRows& q) {
  T o[6], ym[5], yp[5], zm[5], zp[5], wm[5], wp[5];
  quad_row6(x, q, 0, o);
  quad_row_up(x, q, q.py, yp);
  quad_row_down(x, q, -q.py, ym);
  quad_row_up(x, q, q.pz, zp);
  quad_row_down(x, q, -q.pz, zm);
  quad_row_up(x, q, q.py + q.pz, wp);
  quad_row_down(x, q, -q.py - q.pz, wm);
  QuadField<T> f;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    f.ctr[n] = o[n + 1];
    f.nb6[n] = ((o[n] + o[n + 2]) + (ym[n + 1] + yp[n])) + (zm[n + 1] + zp[n]);
    f.d[n].e1 = o[n + 2] - o[n];
    f.d[n].e2 = yp[n] - ym[n + 1];
    f.d[n].e3 = zp[n] - zm[n + 1];
    f.d[n].f12 = yp[n + 1] - ym[n];
    f.d[n].f23 = wp[n] - wm[n + 1];
    f.d[n].f13 = zp[n + 1] - zm[n];
    f.d[n].b = wp[n + 1] - wm[n];
  }
  return f;
}

template <class T>
__global__ void __launch_bounds__(FX * FY) k_residual_quad(LevelDev<T> L) {
  pdl_enter();
  const int pos = blockIdx.x * FX + threadIdx.x;
  const int j = blockIdx.y * FY + threadIdx.y;
  const int k = blockIdx.z;
  const int i0 = 4 * pos - 1;  // lattice x of the quad's first node
  if (j >= L.ny || i0 >= L.nx) return;
  QuadRows q;
  q.g = L.px >> 2;
  q.c = (int64_t)pos + L.px * (j + 1) + L.pxy * (k + 1);
  q.py = L.px;
  q.pz = L.pxy;
  bool fast = i0 >= 0 && i0 + 3 < L.nx;
  uint8_t fl[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    fl[n] = fast ? L.flags[q.c + n * q.g] : (uint8_t)0;
    fast = fast && (fl[n] & (F_ACT | F_VFREE | F_IRR)) == (F_ACT | F_VFREE);
  }
  if (!fast) {
    for (int n = 0; n < 4; ++n) {
      if (i0 + n < 0 || i0 + n >= L.nx) continue;
      node_residual<T, 0>(L, node_at(L.px, L.pxy, i0 + n, j, k));
    }
    return;
  }
  T ru[3][4], rp[4];
  {
    const QuadField<T> p = quad_field(L.p, q);
    const T s = -L.h2 * (T)(1.0 / 12.0);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      T dv[3];
      div12_all(p.d[n], dv);
#pragma unroll
      for (int d = 0; d < 3; ++d) ru[d][n] = L.f[d][q.c + n * q.g] - s * dv[d];
      rp[n] = L.g[q.c + n * q.g] + L.c * ((T)6 * p.ctr[n] - p.nb6[n]);
    }
  }
  T dsum[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const QuadField<T> u = quad_field(L.u[d], q);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      ru[d][n] -= L.nuh * ((T)6 * u.ctr[n] - u.nb6[n]);
      dsum[n] += div12(u.d[n], d);
    }
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int64_t c = q.c + n * q.g;
#pragma unroll
    for (int d = 0; d < 3; ++d) L.r[d][c] = ru[d][n];
    L.rp[c] = rp[n] - L.h2 * (T)(1.0 / 12.0) * dsum[n];
  }
}

template <class T>
__global__ void k_restrict(LevelDev<T> Lf, LevelDev<T> Lc) {
  pdl_enter();
  int i, j, k;
  if (!full_node(Lc, i, j, k)) return;
  node_restrict(Lf, Lc, i, j, k);
}

template <class T>
__global__ void k_prolong_add(LevelDev<T> Lf, LevelDev<T> Lc) {
  pdl_enter();
  int i, j, k;
  if (!full_node(Lf, i, j, k)) return;
  node_prolong_add(Lf, Lc, i, j, k);
}

// ---- reductions ---------------------------------------------------------------

template <int W>
__device__ __forceinline__ void block_reduce_store(double (&v)[W], double* out) {
  __shared__ double sh[W][REDUCE_THREADS / 32];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    double x = v[w];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[w][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double acc = 0;
      for (int q = 0; q < REDUCE_THREADS / 32; ++q) acc += sh[w][q];
      out[w * gridDim.x + blockIdx.x] = acc;
    }
  }
}

template <int W>
__global__ void k_final_sum(const double* partial, int nblocks, double* out) {
  pdl_enter();
  __shared__ double sh[W][32];
  const int lane = threadIdx.x;  // 32 threads
#pragma unroll
  for (int w = 0; w < W; ++w) {
    double acc = 0;
    for (int b = lane; b < nblocks; b += 32) acc += partial[w * nblocks + b];
    sh[w][lane] = acc;
  }
  __syncwarp();
  if (lane == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double acc = 0;
      for (int q = 0; q < 32; ++q) acc += sh[w][q];
      out[w] = acc;
    }
  }
}

template <class T>
__global__ void k_residual_norm2(LevelDev<T> L, double* partial) {
  pdl_enter();
  double v[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L.nalloc; q += stride) {
    const double a = (double)L.r[0][q], b = (double)L.r[1][q], c = (double)L.r[2][q], d = (double)L.rp[q];
    v[0] += (a * a + b * b) + (c * c + d * d);
  }
  block_reduce_store<1>(v, partial);
}

template <class T>
__global__ void k_mass_moments(LevelDev<T> L, double* partial) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) {
    const int i = (int)(q % L.nx);
    const int j = (int)((q / L.nx) % L.ny);
    const int k = (int)(q / ((int64_t)L.nx * L.ny));
    const int64_t c = pidx(L.px, L.pxy, i, j, k);
    const uint8_t fl = L.flags[c];
    if (!(fl & F_ACT)) continue;
    const double m = (double)lumped_mass(L, c, fl);
    v[0] += m * (double)L.p[c];
    v[1] += m;
  }
  block_reduce_store<2>(v, partial);
}

template <class T>
__global__ void k_project(LevelDev<T> L, const double* mom) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const int64_t c = pidx(L.px, L.pxy, i, j, k);
  if (!(L.flags[c] & F_ACT)) return;
  L.p[c] -= (T)(mom[0] / mom[1]);
}

// ---- right-hand side and its transpose (FP64) ------------------------------------

// (M x)_node on a regular node: h^3 [2/5 x_c + 1/20 (axis and body neighbours) + 1/30 (face diagonals)].
__device__ __forceinline__ double mass_reg(const double* x, const Node& n, int64_t px, int64_t pxy, double h3) {
  const GNb<double> v = gnb(x, n, px, pxy);
  const double ax = nb6v(v) + (v(1, 1, 1) + v(-1, -1, -1));
  const double fc = (v(1, 1, 0) + v(-1, -1, 0)) + (v(0, 1, 1) + v(0, -1, -1)) + (v(1, 0, 1) + v(-1, 0, -1));
  return h3 * (0.4 * v(0, 0, 0) + 0.05 * ax + fc * (1.0 / 30.0));
}

__global__ void k_sum_g(LevelDev<double> L, double* partial) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L.nalloc; q += stride) {
    if (L.flags[q] & F_ACT) {
      v[0] += L.g[q];
      v[1] += 1.0;
    }
  }
  block_reduce_store<2>(v, partial);
}

__global__ void k_sub_mean_g(LevelDev<double> L, const double* s) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double mean = s[0] / s[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L.nalloc; q += stride)
    if (L.flags[q] & F_ACT) L.g[q] -= mean;
}

// grad_f_d = M lam_u,d + delta h_T^2 B_d lam_p on active nodes (transpose of
// the right-hand side map f -> (M f, sum_d G_d f_d), with G_d = delta h_T^2 B_d^T).
__global__ void k_rhs_transpose(LevelDev<double> L, double* o0, double* o1, double* o2) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const Node n = node_at(L.px, L.pxy, i, j, k);
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  double* out[3] = {o0, o1, o2};
  if (!(fl & F_ACT)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d][c] = 0.0;
    return;
  }
  const bool irr = fl & F_IRR;
  double bl[3];
  if (!irr) {
    const Diff7<double> dl = diff7(L.p, n, L.px, L.pxy);
    div12_all(dl, bl);
#pragma unroll
    for (int d = 0; d < 3; ++d) bl[d] *= L.h2 * (1.0 / 12.0);
  } else {
    irr_B_scalar(L, L.p, n, bl);
  }
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const double mu = irr ? irr_mass_row(L, L.u[d], n) : mass_reg(L.u[d], n, L.px, L.pxy, L.h3);
    out[d][c] = mu + L.dh2 * bl[d];
  }
}

// ---- mixed precision -------------------------------------------------------------------

__global__ void k_ir_residual(LevelDev<double> X, LevelDev<float> E, double* partial) {
  pdl_enter();
  double v[1] = {0.0};
  const int64_t n = (int64_t)X.nx * X.ny * X.nz;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) {
    const int i = (int)(q % X.nx);
    const int j = (int)((q / X.nx) % X.ny);
    const int k = (int)(q / ((int64_t)X.nx * X.ny));
    const Node n = node_at(X.px, X.pxy, i, j, k);
    const int64_t c = n.c;
    const uint8_t fl = X.flags[c];
    const double* uu[3] = {X.u[0], X.u[1], X.u[2]};  // no address of kernel-parameter members
    if (fl & F_VFREE) {
      double au[3], bt[3];
      row_A(X, uu, n, fl, au);
      row_BT(X, X.p, n, fl, bt);
      double r[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) r[d] = X.f[d][c] - au[d] - bt[d];
      if (fl & F_SLIP) slip_project(class_row(X, c), r);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        E.f[d][c] = (float)r[d];
        v[0] += r[d] * r[d];
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) E.f[d][c] = 0.f;
    }
    if (fl & F_ACT) {
      const double r = X.g[c] - row_B(X, uu, n, fl) + row_C(X, X.p, n, fl);
      E.g[c] = (float)r;
      v[0] += r * r;
    } else {
      E.g[c] = 0.f;
    }
  }
  block_reduce_store<1>(v, partial);
}

// ---- the refinement residual in 64-bit fixed point ------------------------------
// On GB300 an FP64 operation costs about 58 FP32 or integer operations, and
// the FP64 residual of a regular node takes about 130 of them.  Its stencils
// are integer combinations of the iterate (the 7-point Laplacian for A and
// C, twelve times the divergence differences for B and B^T), so they are
// evaluated exactly in 64-bit integers on the iterate quantized per field to
// X = round(x 2^e), with 2^e the power of two that puts max |x| just below
// 2^55: every sum stays below 2^62.  The quantization error is at most
// 2^-56 max |x| per value, of the order of the rounding of the FP64
// evaluation itself.  Each stencil result then takes one conversion and one
// fused multiply-add in FP64 (its scale folded into the operator constant).
// Boundary nodes (class rows) keep the FP64 evaluation.

// max |x| of u_0, u_1, u_2, p as bit patterns of non-negative doubles, which
// order like unsigned integers; mx[0..3] start at zero.
__global__ void k_ir_absmax(LevelDev<double> X, unsigned long long* mx) {
  pdl_enter();
  __shared__ double sh[4][REDUCE_THREADS / 32];
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < X.nalloc; q += stride) {
#pragma unroll
    for (int d = 0; d < 3; ++d) m[d] = fmax(m[d], fabs(X.u[d][q]));
    m[3] = fmax(m[3], fabs(X.p[q]));
  }
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    double x = m[w];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sh[w][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0.0;
    for (int q = 0; q < REDUCE_THREADS / 32; ++q) x = fmax(x, sh[threadIdx.x][q]);
    atomicMax(&mx[threadIdx.x], (unsigned long long)__double_as_longlong(x));
  }
}

// Scale 2^s of a field of the fixed-point iterate from its max |x|: max |x|
// 2^s < 2^(55 - FX_HEADROOM), s capped so that 2^s stays finite; a zero field
// gets the largest scale, so that any nonzero correction of it is refused by
// fx_delta and taken by the host's FP64 path.
constexpr int FX_HEADROOM = 2;
constexpr int FX_ZERO_SHIFT = 995;
__device__ __forceinline__ int fx_shift(unsigned long long bits) {
  const double m = __longlong_as_double((long long)bits);
  if (!(m > 0.0)) return FX_ZERO_SHIFT;
  int E;
  frexp(m, &E);  // m < 2^E
  return 55 - FX_HEADROOM - max(E, -940);
}

// Q = round(x 2^s) per field, s = fx_shift(max |x|) written to fexp; the
// three velocity components share the shift of the largest of them (their
// stencil sums then combine in integers before one conversion).
__global__ void k_ir_quantize(LevelDev<double> X, FxIterate Q, const unsigned long long* mx, int* fexp) {
  pdl_enter();
  double s[4];
  // maxima are FP64 bits of non-negative values: their integer order is theirs
  const unsigned long long mu = max(max(mx[0], mx[1]), mx[2]);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int e = fx_shift(f < 3 ? mu : mx[3]);
    s[f] = ldexp(1.0, e);
    if (blockIdx.x == 0 && threadIdx.x == 0) fexp[f] = e;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < X.nalloc; q += stride) {
#pragma unroll
    for (int d = 0; d < 3; ++d) Q.u[d][q] = __double2ll_rn(X.u[d][q] * s[d]);
    Q.p[q] = __double2ll_rn(X.p[q] * s[3]);
  }
}

// d = round(e 2^s) (halves away from zero) from the bits of e, in integer
// arithmetic; false (d = 0) when |d| could reach 2^57 or e is not finite.
__device__ __forceinline__ bool fx_delta(float e, int s, int64_t& d) {
  const uint32_t b = __float_as_uint(e);
  const int ex = (int)((b >> 23) & 255u);
  uint32_t m = b & 0x7fffffu;
  d = 0;
  if (ex == 255) return false;
  int sh = s - 149;  // e = m 2^(ex - 150) with the leading bit, m 2^-149 without
  if (ex != 0) {
    m |= 0x800000u;
    sh += ex - 1;
  }
  if (m == 0) return true;
  uint64_t a;
  if (sh >= 0) {
    if (sh + (32 - __clz(m)) > 57) return false;
    a = (uint64_t)m << sh;
  } else {
    const int r = -sh;
    if (r > 24) return true;  // m 2^-r < 1/2
    a = ((uint64_t)m + (1ull << (r - 1))) >> r;
  }
  d = (b >> 31) ? -(int64_t)a : (int64_t)a;
  return true;
}

// Q += round(e 2^s) on every padded position, max |Q| per field into maxq
// (zeroed before); a correction fx_delta refuses leaves Q and raises
// FX_FLAG_REFUSED in *flag.
__global__ void k_fx_update(FxIterate Q, LevelDev<float> E, const int* fexp, unsigned long long* maxq,
                            unsigned* flag, int64_t n) {
  pdl_enter();
  __shared__ unsigned long long sh[4][32];
  int s[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) s[f] = fexp[f];
  unsigned long long m[4] = {0, 0, 0, 0};
  bool refused = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int64_t* q = f < 3 ? Q.u[f] : Q.p;
      const float e = f < 3 ? E.u[f][c] : E.p[c];
      int64_t d;
      if (!fx_delta(e, s[f], d)) {
        refused = true;
        continue;
      }
      const int64_t v = q[c] + d;
      q[c] = v;
      m[f] = max(m[f], (unsigned long long)(v < 0 ? -v : v));
    }
  }
  if (refused) atomicOr(flag, FX_FLAG_REFUSED);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    unsigned long long x = m[f];
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) sh[f][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = max(x, sh[threadIdx.x][w]);
    atomicMax(&maxq[threadIdx.x], x);
  }
}

// FP64 iterate from the fixed-point one: x = Q 2^-s, or (recover) the
// iterate before the last k_fx_update plus the FP32 correction in FP64,
// x = (Q - round(e 2^s)) 2^-s + e, with Q untouched where that update
// refused the correction.
__global__ void k_fx_to_fp64(LevelDev<double> X, FxIterate Q, LevelDev<float> E, const int* fexp, int recover) {
  pdl_enter();
  int s[4];
  double is[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    s[f] = fexp[f];
    is[f] = ldexp(1.0, -s[f]);
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < X.nalloc; c += stride) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int64_t q = (f < 3 ? Q.u[f] : Q.p)[c];
      double v;
      if (recover) {
        const float e = f < 3 ? E.u[f][c] : E.p[c];
        int64_t d;
        if (fx_delta(e, s[f], d)) q -= d;
        v = (double)q * is[f] + (double)e;
      } else {
        v = (double)q * is[f];
      }
      (f < 3 ? X.u[f] : X.p)[c] = v;
    }
  }
}

// Slot of a Kuhn neighbour offset in the class-row order: 0 centre, 1..7
// +o, 8..14 -o over e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3.
__host__ __device__ constexpr int kuhn_slot(int dx, int dy, int dz) {
  return (dx | dy | dz) == 0 ? 0
                             : (dx && dy && dz ? 7
                                : dx && dz   ? 6
                                : dy && dz   ? 5
                                : dx && dy   ? 4
                                : dz         ? 3
                                : dy         ? 2
                                             : 1) +
                                   ((dx | dy | dz) < 0 ? 7 : 0);
}
static_assert(kuhn_slot(1, 0, 0) == 1 && kuhn_slot(0, 1, 0) == 2 && kuhn_slot(0, 0, 1) == 3 &&
                  kuhn_slot(1, 1, 0) == 4 && kuhn_slot(0, 1, 1) == 5 && kuhn_slot(1, 0, 1) == 6 &&
                  kuhn_slot(1, 1, 1) == 7 && kuhn_slot(-1, 0, 0) == 8 && kuhn_slot(0, -1, -1) == 12 &&
                  kuhn_slot(-1, -1, -1) == 14 && kuhn_slot(0, 0, 0) == 0,
              "class-row offset order");

// Neighbour view over the 15 values of a node's stencil held in registers.
struct SlotNb {
  const double* v;
  __device__ __forceinline__ double operator()(int dx, int dy, int dz) const { return v[kuhn_slot(dx, dy, dz)]; }
};

// Loads the 15 stencil values of a fixed-point field at node n as FP64 (q 2^-s).
__device__ __forceinline__ void fx_gather15(const int64_t* x, const Node& n, int64_t px, int64_t pxy, double sc,
                                            double v[15]) {
  const GNb<int64_t> g = gnb(x, n, px, pxy);
  v[0] = sc * (double)g(0, 0, 0);
  v[1] = sc * (double)g(1, 0, 0);
  v[2] = sc * (double)g(0, 1, 0);
  v[3] = sc * (double)g(0, 0, 1);
  v[4] = sc * (double)g(1, 1, 0);
  v[5] = sc * (double)g(0, 1, 1);
  v[6] = sc * (double)g(1, 0, 1);
  v[7] = sc * (double)g(1, 1, 1);
  v[8] = sc * (double)g(-1, 0, 0);
  v[9] = sc * (double)g(0, -1, 0);
  v[10] = sc * (double)g(0, 0, -1);
  v[11] = sc * (double)g(-1, -1, 0);
  v[12] = sc * (double)g(0, -1, -1);
  v[13] = sc * (double)g(-1, 0, -1);
  v[14] = sc * (double)g(-1, -1, -1);
}

// (F, G) - K (U, P) in FP64 from the fixed-point iterate on regular nodes,
// FP32 output, and the partial sums of its squared norm.
// With check, the iterate must have come from k_fx_update: when that update
// refused a correction, or a field's max |Q| reached 2^55 (the stencil sums
// could overflow) or fell below 2^45 (too few bits), the kernel raises
// FX_FLAG_RESCALE and returns without output.
__device__ __forceinline__ bool fx_iterate_fit(const unsigned long long* maxq, unsigned* flag) {
  bool ok = *(volatile unsigned*)flag == 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const unsigned long long m = maxq[f];
    if (m >= (1ull << 55) || (m != 0 && m < (1ull << 45))) ok = false;
  }
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flag, FX_FLAG_RESCALE);
  return ok;
}

// The regular nodes; boundary nodes (F_IRR) are left to k_ir_residual_fx_irr.
// Each block takes an FX x FY tile through IR_FZ consecutive planes, one node
// per thread and plane, blocks in lattice order: a block finds the planes
// k - 1 and k + 1 of its tile among the ones it has just read, and its
// neighbour tiles run beside it (a grid-stride loop over the whole level lets
// the blocks drift apart by many planes and reads every plane about twice
// from DRAM).  The block's partial norm goes to partial[linear block index].
__global__ void __launch_bounds__(FX * FY, 3) k_ir_residual_fx(LevelDev<double> X, FxIterate Q, LevelDev<float> E,
                                                            const int* fexp, const unsigned long long* maxq,
                                                            unsigned* flag, int check, double* partial) {
  pdl_enter();
  if (check && !fx_iterate_fit(maxq, flag)) return;
  double is[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) is[f] = ldexp(1.0, -fexp[f]);
  // one shift for the three velocity components (k_ir_quantize)
  const double kA = X.nuh * is[0], kB = X.h2 * (1.0 / 12.0) * is[0];
  const double kBT = X.h2 * (1.0 / 12.0) * is[3], kC = X.c * is[3];
  double v = 0.0;
  const int i = blockIdx.x * FX + threadIdx.x, j = blockIdx.y * FY + threadIdx.y;
  const int k1 = min(X.nz, (int)(blockIdx.z + 1) * IR_FZ);
  for (int k = blockIdx.z * IR_FZ; k < k1; ++k) {
    if (i >= X.nx || j >= X.ny) break;
    const Node n = node_at(X.px, X.pxy, i, j, k);
    const int64_t c = n.c;
    const uint8_t fl = X.flags[c];
    if (!(fl & F_IRR)) {
      const GNb<int64_t> gu[3] = {gnb(Q.u[0], n, X.px, X.pxy), gnb(Q.u[1], n, X.px, X.pxy),
                                  gnb(Q.u[2], n, X.px, X.pxy)};
      const GNb<int64_t> gp = gnb(Q.p, n, X.px, X.pxy);
      double r[4];
      if (fl & F_VFREE) {
        int64_t ibt[3];
        div12_all(diff7v<int64_t>(gp), ibt);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int64_t ia = 6 * gu[d](0, 0, 0) - nb6v(gu[d]);
          r[d] = (X.f[d][c] - kA * (double)ia) + kBT * (double)ibt[d];
        }
      } else {
        r[0] = r[1] = r[2] = 0.0;
      }
      if (fl & F_ACT) {
        const int64_t ic = 6 * gp(0, 0, 0) - nb6v(gp);
        // 12 B u in integers: |Q| < 2^55 keeps each div12 below 15 2^56
        const int64_t ib = (div12(diff7v<int64_t>(gu[0]), 0) + div12(diff7v<int64_t>(gu[1]), 1)) +
                           div12(diff7v<int64_t>(gu[2]), 2);
        r[3] = (X.g[c] - kB * (double)ib) + kC * (double)ic;
      } else {
        r[3] = 0.0;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        E.f[d][c] = (float)r[d];
        v += r[d] * r[d];
      }
      E.g[c] = (float)r[3];
      v += r[3] * r[3];
    }
  }
  // block sum in a fixed order: warps by shuffles, then the warp sums
  __shared__ double sh[FX * FY / 32];
  const int t = threadIdx.x + FX * threadIdx.y;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < FX * FY / 32; ++w) acc += sh[w];
    partial[blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = acc;
  }
}

dim3 ir_residual_grid(const LevelDev<double>& L) {
  return dim3((L.nx + FX - 1) / FX, (L.ny + FY - 1) / FY, (L.nz + IR_FZ - 1) / IR_FZ);
}

// out[b] = sum of in[b n / G, (b + 1) n / G) for the G blocks, in a fixed
// order (first stage of a deterministic sum of many partials).
__global__ void k_segment_sum(const double* in, int64_t n, double* out) {
  pdl_enter();
  const int64_t lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
  double v[1] = {0.0};
  for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x) v[0] += in[q];
  block_reduce_store<1>(v, out);
}

// The boundary nodes of k_ir_residual_fx, from the list of their lattice
// coordinates ((k << 42) | (j << 21) | i): class rows in FP64 on the
// iterate's values, each neighbour converted once.  Partial norms into
// partial[0 .. gridDim.x).
__global__ void k_ir_residual_fx_irr(LevelDev<double> X, FxIterate Q, LevelDev<float> E, const int* fexp,
                                     const unsigned long long* maxq, unsigned* flag, int check,
                                     const int64_t* irr, int64_t nirr, double* partial) {
  pdl_enter();
  if (check && !fx_iterate_fit(maxq, flag)) return;
  double is[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) is[f] = ldexp(1.0, -fexp[f]);
  double v[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nirr; t += stride) {
    const int64_t e = irr[t];
    const Node n = node_at(X.px, X.pxy, (int)(e & 0x1fffff), (int)((e >> 21) & 0x1fffff), (int)(e >> 42));
    const int64_t c = n.c;
    const uint8_t fl = X.flags[c];
    double uv[3][15], pv[15];
#pragma unroll
    for (int d = 0; d < 3; ++d) fx_gather15(Q.u[d], n, X.px, X.pxy, is[d], uv[d]);
    fx_gather15(Q.p, n, X.px, X.pxy, is[3], pv);
    const SlotNb u[3] = {SlotNb{uv[0]}, SlotNb{uv[1]}, SlotNb{uv[2]}};
    double r[4];
    node_residual_v(X, c, fl, u, SlotNb{pv}, r);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      E.f[d][c] = (float)r[d];
      v[0] += r[d] * r[d];
    }
    E.g[c] = (float)r[3];
    v[0] += r[3] * r[3];
  }
  block_reduce_store<1>(v, partial);
}

// ---- right-hand side in fixed point ------------------------------------------------

// In place: the staged nodal f (a0..a2) and u_D (b0..b2) become int64
// round(v 2^s), one shift for f and one for u_D from their max |v| (mx[0..3)
// and mx[4..7)), written to sh[0..2).
__global__ void k_rhs_quantize(double* a0, double* a1, double* a2, double* b0, double* b1, double* b2,
                               const unsigned long long* mx, int* sh, int64_t n) {
  pdl_enter();
  const int sf = fx_shift(max(max(mx[0], mx[1]), mx[2]));
  const int su = fx_shift(max(max(mx[4], mx[5]), mx[6]));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sh[0] = sf;
    sh[1] = su;
  }
  const double cf = ldexp(1.0, sf), cu = ldexp(1.0, su);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double* a = k == 0 ? a0 : k == 1 ? a1 : k == 2 ? a2 : k == 3 ? b0 : k == 4 ? b1 : b2;
      const double v = a[c];
      reinterpret_cast<int64_t*>(a)[c] = __double2ll_rn(v * (k < 3 ? cf : cu));
    }
  }
}

// f~ = M f - A u_D (velocity nodes), g~ = delta h_T^2 sum_d B_d^T f_d - B u_D
// (pressure nodes) on the regular nodes from the quantized data: the mass,
// stiffness and divergence stencils as exact integer sums (60 M_reg / h^3 =
// 24 centre + 3 axis/body + 2 face diagonals), one conversion per term.
// Boundary nodes are left to k_set_rhs_irr.
__global__ void k_set_rhs_fx(LevelDev<double> L, const int64_t* f0, const int64_t* f1, const int64_t* f2,
                             const int64_t* d0, const int64_t* d1, const int64_t* d2, const int* sh) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const Node n = node_at(L.px, L.pxy, i, j, k);
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  if (fl & F_IRR) return;
  const double isf = ldexp(1.0, -sh[0]), isu = ldexp(1.0, -sh[1]);
  const GNb<int64_t> F[3] = {gnb(f0, n, L.px, L.pxy), gnb(f1, n, L.px, L.pxy), gnb(f2, n, L.px, L.pxy)};
  const GNb<int64_t> U[3] = {gnb(d0, n, L.px, L.pxy), gnb(d1, n, L.px, L.pxy), gnb(d2, n, L.px, L.pxy)};
  if (fl & F_VFREE) {
    const double km = L.h3 * (1.0 / 60.0) * isf, ka = L.nuh * isu;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const GNb<int64_t>& v = F[d];
      const int64_t ax = nb6v(v) + (v(1, 1, 1) + v(-1, -1, -1));
      const int64_t fc = (v(1, 1, 0) + v(-1, -1, 0)) + (v(0, 1, 1) + v(0, -1, -1)) + (v(1, 0, 1) + v(-1, 0, -1));
      const int64_t m = 24 * v(0, 0, 0) + 3 * ax + 2 * fc;
      const int64_t a = 6 * U[d](0, 0, 0) - nb6v(U[d]);
      L.f[d][c] = km * (double)m - ka * (double)a;
    }
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) L.f[d][c] = 0.0;
  }
  if (fl & F_ACT) {
    const int64_t bf = (div12(diff7v<int64_t>(F[0]), 0) + div12(diff7v<int64_t>(F[1]), 1)) +
                       div12(diff7v<int64_t>(F[2]), 2);
    const int64_t bu = (div12(diff7v<int64_t>(U[0]), 0) + div12(diff7v<int64_t>(U[1]), 1)) +
                       div12(diff7v<int64_t>(U[2]), 2);
    const double k12 = L.h2 * (1.0 / 12.0);
    L.g[c] = (L.dh2 * (-k12 * isf)) * (double)bf - (k12 * isu) * (double)bu;
  } else {
    L.g[c] = 0.0;
  }
}

// The boundary nodes (list of lattice coordinates, as k_ir_residual_fx_irr):
// class rows in FP64 on the dequantized data, component by component.
__global__ void k_set_rhs_irr(LevelDev<double> L, const int64_t* f0, const int64_t* f1, const int64_t* f2,
                              const int64_t* d0, const int64_t* d1, const int64_t* d2, const int* sh,
                              const int64_t* irr, int64_t nirr) {
  pdl_enter();
  const double isf = ldexp(1.0, -sh[0]), isu = ldexp(1.0, -sh[1]);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nirr; t += stride) {
    const int64_t e = irr[t];
    const Node n = node_at(L.px, L.pxy, (int)(e & 0x1fffff), (int)((e >> 21) & 0x1fffff), (int)(e >> 42));
    const int64_t c = n.c;
    const uint8_t fl = L.flags[c];
    const double* w = class_row(L, c);
    double gf = 0.0, gu = 0.0;
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      double fv[15], uv[15];
      fx_gather15(d == 0 ? f0 : d == 1 ? f1 : f2, n, L.px, L.pxy, isf, fv);
      fx_gather15(d == 0 ? d0 : d == 1 ? d1 : d2, n, L.px, L.pxy, isu, uv);
      const SlotNb fs{fv}, us{uv};
      if (fl & F_VFREE) L.f[d][c] = L.h3 * st15v<double>(fs, w + W_M) - L.nuh * st15v<double>(us, w + W_LAP);
      gf += L.h2 * st15v<double>(fs, w + W_BT + 15 * d);
      gu += st15v<double>(us, w + W_B + 15 * d);
    }
    if (!(fl & F_VFREE)) {
#pragma unroll
      for (int d = 0; d < 3; ++d) L.f[d][c] = 0.0;
    }
    L.g[c] = (fl & F_ACT) ? L.dh2 * gf - L.h2 * gu : 0.0;
  }
}

// D form: f_a += nu h (A1 u_D)_a - nu h (A2 u_D)_a on velocity nodes, from the
// quantized staged u_D (the values launch_set_rhs lifted with).
__global__ void k_lift_d(LevelDev<double> L, const int64_t* d0, const int64_t* d1, const int64_t* d2,
                         const int* sh) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const Node n = node_at(L.px, L.pxy, i, j, k);
  const uint8_t fl = L.flags[n.c];
  if (!(fl & F_VFREE)) return;
  const double isu = ldexp(1.0, -sh[1]);
  double uv[3][15];
  fx_gather15(d0, n, L.px, L.pxy, isu, uv[0]);
  fx_gather15(d1, n, L.px, L.pxy, isu, uv[1]);
  fx_gather15(d2, n, L.px, L.pxy, isu, uv[2]);
  const SlotNb u[3] = {SlotNb{uv[0]}, SlotNb{uv[1]}, SlotNb{uv[2]}};
  double a2[3], a1[3];
  row_A2_v(L, u, d_row(L, n.c), a2);
  row_A_v(L, u, row_of(L, n.c, fl), fl, a1);
#pragma unroll
  for (int d = 0; d < 3; ++d) L.f[d][n.c] += a1[d] - a2[d];
}

// x += e (the FP64 refinement update).
__global__ void k_ir_update(LevelDev<double> X, LevelDev<float> E) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < X.nalloc; q += stride) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X.u[d][q] += (double)E.u[d][q];
    X.p[q] += (double)E.p[q];
  }
}

// Free slip (Sec. 6.1): after a refinement update the velocity of every
// slip node of the boundary list is made tangential again in FP64 (the FP32
// correction is tangential only to FP32 rounding, and a normal part would
// reach the pressure rows through B).  FP64 iterate:
__global__ void k_slip_fix(LevelDev<double> X, const int64_t* irr, int64_t nirr) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nirr; t += stride) {
    const int64_t e = irr[t];
    const int64_t c = pidx(X.px, X.pxy, (int)(e & 0x1fffff), (int)((e >> 21) & 0x1fffff), (int)(e >> 42));
    if (!(X.flags[c] & F_SLIP)) continue;
    double v[3] = {X.u[0][c], X.u[1][c], X.u[2][c]};
    slip_project(class_row(X, c), v);
#pragma unroll
    for (int d = 0; d < 3; ++d) X.u[d][c] = v[d];
  }
}

// The same on the fixed-point iterate (the three velocity fields share one
// shift, so the projection acts on Q directly); a value that leaves the
// range the fixed-point checks allow raises FX_FLAG_RESCALE (the host then
// rebuilds and requantizes the FP64 iterate).
__global__ void k_slip_fix_fx(FxIterate Q, LevelDev<double> X, const int64_t* irr, int64_t nirr, unsigned* flag) {
  pdl_enter();
  bool big = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nirr; t += stride) {
    const int64_t e = irr[t];
    const int64_t c = pidx(X.px, X.pxy, (int)(e & 0x1fffff), (int)((e >> 21) & 0x1fffff), (int)(e >> 42));
    if (!(X.flags[c] & F_SLIP)) continue;
    double v[3] = {(double)Q.u[0][c], (double)Q.u[1][c], (double)Q.u[2][c]};
    slip_project(class_row(X, c), v);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long q = llrint(v[d]);
      big |= (q < 0 ? -q : q) >= (1ll << 55);
      Q.u[d][c] = q;
    }
  }
  if (big) atomicOr(flag, FX_FLAG_RESCALE);
}

// ---- layout conversion ---------------------------------------------------------------------

__global__ void k_scatter(LevelDev<double> L, const double* src, int ncomp, double* d0, double* d1, double* d2,
                          uint8_t mask) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const int64_t c = pidx(L.px, L.pxy, i, j, k);
  const int64_t q = i + (int64_t)L.nx * (j + (int64_t)L.ny * k);
  const bool keep = mask == 0 || (L.flags[c] & mask);
  double* dst[3] = {d0, d1, d2};
  for (int d = 0; d < ncomp; ++d) dst[d][c] = keep ? src[ncomp * q + d] : 0.0;
}

template <class T>
__global__ void k_gather(LevelDev<T> L, const T* s0, const T* s1, const T* s2, int ncomp, double* dst) {
  pdl_enter();
  int i, j, k;
  if (!full_node(L, i, j, k)) return;
  const int64_t c = pidx(L.px, L.pxy, i, j, k);
  const int64_t q = i + (int64_t)L.nx * (j + (int64_t)L.ny * k);
  const T* src[3] = {s0, s1, s2};
  for (int d = 0; d < ncomp; ++d) dst[ncomp * q + d] = (double)src[d][c];
}

__global__ void k_dirichlet_fill(const int64_t* idx, const double* val, int64_t ndir, double* dst) {
  pdl_enter();
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= ndir) return;
  const int64_t n = idx[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) dst[3 * n + d] = val[3 * q + d];
}

__global__ void k_dirichlet_gather(const int64_t* pad, int64_t ndir, const double* u0, const double* u1,
                                   const double* u2, double* val) {
  pdl_enter();
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= ndir) return;
  const int64_t c = pad[q];
  val[3 * q + 0] = u0[c];
  val[3 * q + 1] = u1[c];
  val[3 * q + 2] = u2[c];
}

// Nodal data of a coarser level taken at its nodes from the finest level's
// padded arrays (node (i, j, k) of the coarse level is node (s i, s j, s k) of
// the finest): body force into RU on active nodes, Dirichlet data into U on
// Dirichlet nodes, zero elsewhere (the layout hhg_set_rhs stages).
__global__ void k_inject(LevelDev<double> Lf, LevelDev<double> Lc, int s) {
  pdl_enter();
  int i, j, k;
  if (!full_node(Lc, i, j, k)) return;
  const int64_t cc = pidx(Lc.px, Lc.pxy, i, j, k);
  const int64_t cf = pidx(Lf.px, Lf.pxy, s * i, s * j, s * k);
  const uint8_t fl = Lc.flags[cc];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Lc.r[d][cc] = (fl & F_ACT) ? Lf.r[d][cf] : 0.0;
    Lc.u[d][cc] = (fl & F_DIR) ? Lf.u[d][cf] : 0.0;
  }
}

// U at the listed (padded) Dirichlet nodes = their values (3 per node).
__global__ void k_dirichlet_scatter(const int64_t* pad, int64_t ndir, const double* val, double* u0, double* u1,
                                    double* u2) {
  pdl_enter();
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= ndir) return;
  const int64_t c = pad[q];
  u0[c] = val[3 * q + 0];
  u1[c] = val[3 * q + 1];
  u2[c] = val[3 * q + 2];
}

__global__ void k_scale(double* x, int64_t n, double a) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) x[q] *= a;
}

__global__ void k_cast(const double* src, float* dst, int64_t n) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) dst[q] = (float)src[q];
}

// Launch with programmatic stream serialization (see pdl_enter).
template <class... KArgs, class... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

int flat_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

// ---- launchers -------------------------------------------------------------------------

template <class T>
void launch_vel_rhs(const LevelDev<T>& L, cudaStream_t s) {
  launch_k(k_vel_rhs<T>, full_grid(L), dim3(FX, FY), s, L);
}
template <class T>
void launch_vel_colour(const LevelDev<T>& L, int colour, cudaStream_t s) {
  const T inv = (T)(1.0 / (6.0 * (double)L.nuh));
  const bool sp = spec_level(L), df = L.wt2 != nullptr;
  if (sp && df)
    launch_k(k_vel_colour<T, true, 1>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else if (sp)
    launch_k(k_vel_colour<T, true, 0>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else if (df)
    launch_k(k_vel_colour<T, false, 1>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else
    launch_k(k_vel_colour<T, false, 0>, colour_grid(L), colour_block(L), s, L, colour, inv);
}
template <class T>
void launch_vel_colour_rhs(const LevelDev<T>& L, int colour, cudaStream_t s) {
  const T inv = (T)(1.0 / (6.0 * (double)L.nuh));
  if constexpr (std::is_same<T, float>::value) {
    if (L.pairs) {
      launch_k(k_colour_pair<0>, pair_grid(L), colour_block(L), s, L, colour, inv, 0.0f);
      return;
    }
  }
  const bool sp = spec_level(L), df = L.wt2 != nullptr;
  if (sp && df)
    launch_k(k_vel_colour_rhs<T, true, 1>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else if (sp)
    launch_k(k_vel_colour_rhs<T, true, 0>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else if (df)
    launch_k(k_vel_colour_rhs<T, false, 1>, colour_grid(L), colour_block(L), s, L, colour, inv);
  else
    launch_k(k_vel_colour_rhs<T, false, 0>, colour_grid(L), colour_block(L), s, L, colour, inv);
}
template <class T>
void launch_vel_pres_colour0(const LevelDev<T>& L, bool ru, cudaStream_t s) {
  const T inv = (T)(1.0 / (6.0 * (double)L.nuh));
  const T w = (T)((double)L.omega / (6.0 * (double)L.c));
  const bool sp = spec_level(L);
  if constexpr (std::is_same<T, float>::value) {
    if (L.pairs && !ru) {
      launch_k(k_colour_pair<2>, pair_grid(L), colour_block(L), s, L, 0, inv, w);
      return;
    }
  }
  auto go = [&](auto kernel) { launch_k(kernel, colour_grid(L), colour_block(L), s, L, inv, w); };
  if (L.wt2) {
    if (ru && sp)
      go(k_vel_pres_colour0<T, true, true, 1>);
    else if (ru)
      go(k_vel_pres_colour0<T, true, false, 1>);
    else if (sp)
      go(k_vel_pres_colour0<T, false, true, 1>);
    else
      go(k_vel_pres_colour0<T, false, false, 1>);
  } else {
    if (ru && sp)
      go(k_vel_pres_colour0<T, true, true, 0>);
    else if (ru)
      go(k_vel_pres_colour0<T, true, false, 0>);
    else if (sp)
      go(k_vel_pres_colour0<T, false, true, 0>);
    else
      go(k_vel_pres_colour0<T, false, false, 0>);
  }
}

template <class T>
void launch_pres_colour_rhs(const LevelDev<T>& L, int colour, cudaStream_t s) {
  const T w = (T)((double)L.omega / (6.0 * (double)L.c));
  if constexpr (std::is_same<T, float>::value) {
    if (L.pairs) {
      launch_k(k_colour_pair<1>, pair_grid(L), colour_block(L), s, L, colour, 0.0f, w);
      return;
    }
  }
  if (spec_level(L))
    launch_k(k_pres_colour_rhs<T, true>, colour_grid(L), colour_block(L), s, L, colour, w);
  else
    launch_k(k_pres_colour_rhs<T, false>, colour_grid(L), colour_block(L), s, L, colour, w);
}
template <class T>
void launch_pres_rhs(const LevelDev<T>& L, cudaStream_t s) {
  launch_k(k_pres_rhs<T>, full_grid(L), dim3(FX, FY), s, L);
}
template <class T>
void launch_pres_colour(const LevelDev<T>& L, int colour, cudaStream_t s) {
  const T w = (T)((double)L.omega / (6.0 * (double)L.c));
  launch_k(k_pres_colour<T>, colour_grid(L), colour_block(L), s, L, colour, w);
}
template <class T>
void launch_residual(const LevelDev<T>& L, cudaStream_t s) {
  if (L.wt2) {
    launch_k(k_residual<T, 1>, full_grid(L), dim3(FX, FY), s, L);
  } else if (L.quad) {
    const int npos = L.nx / 4 + 1;  // quads cover padded x = 0 .. 4 npos - 1 >= nx
    launch_k(k_residual_quad<T>, dim3((npos + FX - 1) / FX, (L.ny + FY - 1) / FY, L.nz), dim3(FX, FY), s, L);
  } else {
    launch_k(k_residual<T, 0>, full_grid(L), dim3(FX, FY), s, L);
  }
}
template <class T>
void launch_restrict(const LevelDev<T>& fine, const LevelDev<T>& coarse, cudaStream_t s) {
  launch_k(k_restrict<T>, full_grid(coarse), dim3(FX, FY), s, fine, coarse);
}
template <class T>
void launch_prolong_add(const LevelDev<T>& fine, const LevelDev<T>& coarse, cudaStream_t s) {
  launch_k(k_prolong_add<T>, full_grid(fine), dim3(FX, FY), s, fine, coarse);
}
template <class T>
void launch_residual_norm2(const LevelDev<T>& L, double* partial, double* out, cudaStream_t s) {
  launch_k(k_residual_norm2<T>, REDUCE_BLOCKS, REDUCE_THREADS, s, L, partial);
  launch_k(k_final_sum<1>, 1, 32, s, partial, REDUCE_BLOCKS, out);
}
template <class T>
void launch_mass_moments(const LevelDev<T>& L, double* partial, double* out, cudaStream_t s) {
  launch_k(k_mass_moments<T>, REDUCE_BLOCKS, REDUCE_THREADS, s, L, partial);
  launch_k(k_final_sum<2>, 1, 32, s, partial, REDUCE_BLOCKS, out);
}
template <class T>
void launch_project(const LevelDev<T>& L, const double* moments, cudaStream_t s) {
  launch_k(k_project<T>, full_grid(L), dim3(FX, FY), s, L, moments);
}
template <class T>
void launch_zero(const LevelDev<T>& L, int what, cudaStream_t s) {
  T* base = what == 0 ? L.u[0] : (what == 1 ? L.f[0] : L.r[0]);
  cudaMemsetAsync(base, 0, sizeof(T) * 4 * (size_t)L.nalloc, s);
}

void launch_set_rhs(const LevelDev<double>& L, double* const* fnod, double* const* uD, unsigned long long* mx,
                    int* sh, const int64_t* irr, int64_t nirr, cudaStream_t s) {
  cudaMemsetAsync(mx, 0, 8 * sizeof(unsigned long long), s);
  LevelDev<double> a = L;  // the max |v| kernel reads u[0..3) and p
  for (int d = 0; d < 3; ++d) a.u[d] = fnod[d];
  a.p = fnod[0];
  launch_k(k_ir_absmax, IR_BLOCKS, REDUCE_THREADS, s, a, mx);
  for (int d = 0; d < 3; ++d) a.u[d] = uD[d];
  a.p = uD[0];
  launch_k(k_ir_absmax, IR_BLOCKS, REDUCE_THREADS, s, a, mx + 4);
  launch_k(k_rhs_quantize, flat_blocks(L.nalloc), 256, s, fnod[0], fnod[1], fnod[2], uD[0], uD[1], uD[2],
           (const unsigned long long*)mx, sh, L.nalloc);
  const int64_t* f[3] = {reinterpret_cast<const int64_t*>(fnod[0]), reinterpret_cast<const int64_t*>(fnod[1]),
                         reinterpret_cast<const int64_t*>(fnod[2])};
  const int64_t* u[3] = {reinterpret_cast<const int64_t*>(uD[0]), reinterpret_cast<const int64_t*>(uD[1]),
                         reinterpret_cast<const int64_t*>(uD[2])};
  launch_k(k_set_rhs_fx, full_grid(L), dim3(FX, FY), s, L, f[0], f[1], f[2], u[0], u[1], u[2], (const int*)sh);
  if (nirr > 0)
    launch_k(k_set_rhs_irr, IR_IRR_BLOCKS, REDUCE_THREADS, s, L, f[0], f[1], f[2], u[0], u[1], u[2],
             (const int*)sh, irr, nirr);
}
void launch_lift_d(const LevelDev<double>& L, double* const* uD, const int* sh, cudaStream_t s) {
  launch_k(k_lift_d, full_grid(L), dim3(FX, FY), s, L, reinterpret_cast<const int64_t*>(uD[0]),
           reinterpret_cast<const int64_t*>(uD[1]), reinterpret_cast<const int64_t*>(uD[2]), sh);
}
void launch_remove_mean_g(const LevelDev<double>& L, double* partial, double* out, cudaStream_t s) {
  launch_k(k_sum_g, REDUCE_BLOCKS, REDUCE_THREADS, s, L, partial);
  launch_k(k_final_sum<2>, 1, 32, s, partial, REDUCE_BLOCKS, out);
  launch_k(k_sub_mean_g, flat_blocks(L.nalloc), 256, s, L, out);
}
void launch_rhs_transpose(const LevelDev<double>& L, double* const* out, cudaStream_t s) {
  launch_k(k_rhs_transpose, full_grid(L), dim3(FX, FY), s, L, out[0], out[1], out[2]);
}
void launch_ir_residual(const LevelDev<double>& x, const LevelDev<float>& e, double* partial, double* out,
                        cudaStream_t s) {
  launch_k(k_ir_residual, REDUCE_BLOCKS, REDUCE_THREADS, s, x, e, partial);
  launch_k(k_final_sum<1>, 1, 32, s, partial, REDUCE_BLOCKS, out);
}
void launch_ir_residual_fx(const LevelDev<double>& x, const FxIterate& q, const LevelDev<float>& e, const FxState& st,
                           bool from_update, double* partial, double* out, cudaStream_t s) {
  if (!from_update) {
    cudaMemsetAsync(st.flag, 0, sizeof(unsigned), s);
    cudaMemsetAsync(st.mx, 0, 4 * sizeof(unsigned long long), s);
    launch_k(k_ir_absmax, IR_BLOCKS, REDUCE_THREADS, s, x, st.mx);
    launch_k(k_ir_quantize, flat_blocks(x.nalloc), 256, s, x, q, (const unsigned long long*)st.mx, st.exp);
  }
  const dim3 grid = ir_residual_grid(x);
  const int64_t nreg = (int64_t)grid.x * grid.y * grid.z;
  launch_k(k_ir_residual_fx, grid, dim3(FX, FY), s, x, q, e, (const int*)st.exp, (const unsigned long long*)st.maxq,
           st.flag, from_update ? 1 : 0, partial);
  launch_k(k_ir_residual_fx_irr, IR_IRR_BLOCKS, REDUCE_THREADS, s, x, q, e, (const int*)st.exp,
           (const unsigned long long*)st.maxq, st.flag, from_update ? 1 : 0, (const int64_t*)st.irr, st.nirr,
           partial + nreg);
  double* seg = partial + nreg + IR_IRR_BLOCKS;
  launch_k(k_segment_sum, IR_BLOCKS, REDUCE_THREADS, s, (const double*)partial, nreg + IR_IRR_BLOCKS, seg);
  launch_k(k_final_sum<1>, 1, 32, s, (const double*)seg, IR_BLOCKS, out);
}
int64_t ir_residual_fx_partials(const LevelDev<double>& x) {
  const dim3 grid = ir_residual_grid(x);
  return (int64_t)grid.x * grid.y * grid.z + IR_IRR_BLOCKS + IR_BLOCKS;
}
void launch_fx_update(const FxIterate& q, const LevelDev<float>& e, const FxState& st, int64_t nalloc, cudaStream_t s) {
  cudaMemsetAsync(st.maxq, 0, 4 * sizeof(unsigned long long), s);
  launch_k(k_fx_update, flat_blocks(nalloc), 256, s, q, e, (const int*)st.exp, st.maxq, st.flag, nalloc);
}
void launch_fx_to_fp64(const LevelDev<double>& x, const FxIterate& q, const LevelDev<float>& e, const FxState& st,
                       bool recover, cudaStream_t s) {
  launch_k(k_fx_to_fp64, flat_blocks(x.nalloc), 256, s, x, q, e, (const int*)st.exp, recover ? 1 : 0);
}

void launch_slip_fix(const LevelDev<double>& x, const int64_t* irr, int64_t nirr, cudaStream_t s) {
  launch_k(k_slip_fix, flat_blocks(nirr), 256, s, x, irr, nirr);
}
void launch_slip_fix_fx(const FxIterate& q, const LevelDev<double>& x, const FxState& st, cudaStream_t s) {
  launch_k(k_slip_fix_fx, flat_blocks(st.nirr), 256, s, q, x, st.irr, st.nirr, st.flag);
}
void launch_ir_update(const LevelDev<double>& x, const LevelDev<float>& e, cudaStream_t s) {
  launch_k(k_ir_update, flat_blocks(x.nalloc), 256, s, x, e);
}
void launch_scatter(const LevelDev<double>& L, const double* src, int ncomp, double* const* dst, uint8_t mask,
                    cudaStream_t s) {
  k_scatter<<<full_grid(L), dim3(FX, FY), 0, s>>>(L, src, ncomp, dst[0], ncomp > 1 ? dst[1] : dst[0],
                                                   ncomp > 2 ? dst[2] : dst[0], mask);
}
template <class T>
void launch_gather(const LevelDev<T>& L, const T* const* src, int ncomp, double* dst, cudaStream_t s) {
  k_gather<T><<<full_grid(L), dim3(FX, FY), 0, s>>>(L, src[0], ncomp > 1 ? src[1] : src[0],
                                                     ncomp > 2 ? src[2] : src[0], ncomp, dst);
}
void launch_dirichlet_fill(const int64_t* idx, const double* val, int64_t ndir, const LevelDev<double>&, double* dst,
                           cudaStream_t s) {
  if (ndir == 0) return;
  launch_k(k_dirichlet_fill, (unsigned)((ndir + 255) / 256), 256, s, idx, val, ndir, dst);
}
void launch_dirichlet_gather(const int64_t* pad, int64_t ndir, const LevelDev<double>& L, double* val,
                             cudaStream_t s) {
  if (ndir == 0) return;
  launch_k(k_dirichlet_gather, (unsigned)((ndir + 255) / 256), 256, s, pad, ndir, L.u[0], L.u[1], L.u[2], val);
}
void launch_scale(double* x, int64_t n, double a, cudaStream_t s) { launch_k(k_scale, flat_blocks(n), 256, s, x, n, a); }
void launch_inject(const LevelDev<double>& fine, const LevelDev<double>& coarse, int stride, cudaStream_t s) {
  launch_k(k_inject, full_grid(coarse), dim3(FX, FY), s, fine, coarse, stride);
}
void launch_dirichlet_scatter(const int64_t* pad, int64_t ndir, const double* val, const LevelDev<double>& L,
                              cudaStream_t s) {
  if (ndir == 0) return;
  launch_k(k_dirichlet_scatter, (unsigned)((ndir + 255) / 256), 256, s, pad, ndir, val, L.u[0], L.u[1], L.u[2]);
}
void launch_cast_field(const double* src, float* dst, int64_t n, cudaStream_t s) {
  launch_k(k_cast, flat_blocks(n), 256, s, src, dst, n);
}

#define HHG_INST(T)                                                                                    \
  template void launch_vel_rhs<T>(const LevelDev<T>&, cudaStream_t);                                    \
  template void launch_vel_colour<T>(const LevelDev<T>&, int, cudaStream_t);                            \
  template void launch_pres_rhs<T>(const LevelDev<T>&, cudaStream_t);                                   \
  template void launch_vel_colour_rhs<T>(const LevelDev<T>&, int, cudaStream_t);                        \
  template void launch_pres_colour_rhs<T>(const LevelDev<T>&, int, cudaStream_t);                       \
  template void launch_vel_pres_colour0<T>(const LevelDev<T>&, bool, cudaStream_t);                      \
  template void launch_pres_colour<T>(const LevelDev<T>&, int, cudaStream_t);                           \
  template void launch_residual<T>(const LevelDev<T>&, cudaStream_t);                                   \
  template void launch_restrict<T>(const LevelDev<T>&, const LevelDev<T>&, cudaStream_t);               \
  template void launch_prolong_add<T>(const LevelDev<T>&, const LevelDev<T>&, cudaStream_t);            \
  template void launch_residual_norm2<T>(const LevelDev<T>&, double*, double*, cudaStream_t);           \
  template void launch_mass_moments<T>(const LevelDev<T>&, double*, double*, cudaStream_t);             \
  template void launch_project<T>(const LevelDev<T>&, const double*, cudaStream_t);                     \
  template void launch_zero<T>(const LevelDev<T>&, int, cudaStream_t);                                  \
  template void launch_gather<T>(const LevelDev<T>&, const T* const*, int, double*, cudaStream_t);

HHG_INST(double)
HHG_INST(float)

}  // namespace hhg
