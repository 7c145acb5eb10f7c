// Device-side level views and stencil arithmetic of the P1-P1 Stokes operator
// on the Kuhn lattice.
//
// Storage: every field of a level is one padded 3-D array over the lattice
// with a zero ghost frame of one node; node (i,j,k) lives at
// pad_index(px, pxy, i, j, k) (rows grouped by x mod 4, hhg_common.h), and a
// Node carries that index with the row steps to its x-neighbours.  Fields
// are zero on nodes without the
// corresponding unknown (velocity: not F_VFREE, pressure: not F_ACT); every
// kernel keeps that invariant, so stencils need no neighbour masks.
//
// Operators (Sec. 2.1 forms on a level with lattice spacing h, |T| = h^3/6,
// h_T = |T|^(1/3)), written through three unit stencils:
//   Lap x = 6 x_c - sum of the 6 axis neighbours       (A = nu h Lap, C = delta h_T^2 h Lap)
//   Div_d x = sum_o s_d(o) (x(c+o) - x(c-o))            (B_d = h^2 Div_d, B_d^T = -h^2 Div_d)
//     over the 7 Kuhn directions o; 12 s_d = -3 on e_d, +1 on the other axes,
//     -1 on the face diagonals containing e_d, +1 on the other, -1 on (1,1,1)
//   mass and g-map for the right-hand side.
// These constant stencils hold on "regular" nodes (all 24 incident
// tetrahedra active).  A node flagged F_IRR belongs to a stencil class (the
// set of its active incident tetrahedra); its rows are 15-point weights from
// a per-level class table assembled at set-up from the element matrices.
#pragma once
#include <stdint.h>

#include "hhg_common.h"

namespace hhg {

template <class T>
struct LevelDev {
  int nx, ny, nz;        // lattice nodes per axis
  int level;             // refinement level (2^level fine cells per macro cell edge)
  int mx, my, mz;        // macro cells per axis
  int64_t px, pxy;       // padded strides
  int64_t nalloc;        // padded entries per field
  const uint8_t* flags;  // padded node flags
  const uint8_t* mmask;  // macro cell masks
  const uint16_t* cls;   // padded stencil class of F_IRR nodes
  const T* wt;           // class table, W_STRIDE weights per class
  const T* wt2;          // D form (Sec. 2.1, a_2): rows of the velocity block, W2_STRIDE per class
                         // (class 0: full-star nodes); null in the Laplace form
  T nuh;                 // nu * h
  T c;                   // delta * h_T^2 * h
  T h2;                  // h^2
  T h3;                  // h^3
  T dh2;                 // delta * h_T^2
  T omega;               // pressure under-relaxation
  int spec;              // colour updates in the speculative node form (small levels)
  int cbz;               // planes per thread block of the colour kernels
  int nq;                // quarter-row slots per row, (nx + 3) / 4: the colour kernels' packed index
  uint64_t nq_mul;       // ceil(2^64 / nq) (0 when nq = 1): t / nq = umul64hi(t, nq_mul)
  int pairs;             // FP32 colour kernels update two nodes per thread (hhg_kernels.cu)
  int quad;              // the residual four nodes per thread (k_residual_quad, Laplace form)
  int nq2;               // pair slots per row, nq / 2 + 1
  uint64_t nq2_mul;      // ceil(2^64 / nq2)
  T* u[3];
  T* p;
  T* f[3];
  T* g;
  T* r[3];
  T* rp;
};

// Programmatic dependent launch: every kernel of the library is launched so
// that the next one may be scheduled while it runs.  A kernel first waits
// until the grid it depends on has completed and its writes are visible
// (griddepcontrol.wait returns at once when there is no such grid), then lets
// its own dependent grid be scheduled; no kernel touches device memory before
// the wait.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ int64_t pidx(int64_t px, int64_t pxy, int i, int j, int k) {
  return pad_index(px, pxy, i, j, k);
}

// A node's padded index and the steps to its x-neighbours within the row.
struct Node {
  int64_t c, dxm, dxp;
};

__device__ __forceinline__ Node node_at(int64_t px, int64_t pxy, int i, int j, int k) {
  return Node{pad_index(px, pxy, i, j, k), row_step_minus(i + 1, px), row_step_plus(i + 1, px)};
}

// ---- neighbour views -----------------------------------------------------------
// V(dx, dy, dz) is a field's value at the node offset by (dx, dy, dz) from the
// node the view is centred on.  The stencil arithmetic below is written once
// over views, so kernels that read the padded arrays in global memory and
// kernels that read a shared-memory tile do the same operations in the same
// order.
//
// GNb: padded array in global memory.  The row helpers read fields that fused
// kernels also write in earlier phases of the same launch, so they use plain
// (coherent) loads.
template <class T>
struct GNb {
  const T* x;
  Node n;
  int64_t px, pxy;
  __device__ __forceinline__ T operator()(int dx, int dy, int dz) const {
    return x[n.c + (dx < 0 ? n.dxm : (dx > 0 ? n.dxp : 0)) + px * dy + pxy * dz];
  }
};

template <class T>
__device__ __forceinline__ GNb<T> gnb(const T* x, const Node& n, int64_t px, int64_t pxy) {
  return GNb<T>{x, n, px, pxy};
}

// Sum of the six axis neighbours.
template <class V>
__device__ __forceinline__ auto nb6v(const V& x) {
  return ((x(-1, 0, 0) + x(1, 0, 0)) + (x(0, -1, 0) + x(0, 1, 0))) + (x(0, 0, -1) + x(0, 0, 1));
}

template <class T>
__device__ __forceinline__ T nb6(const T* x, const Node& n, int64_t px, int64_t pxy) {
  return nb6v(gnb(x, n, px, pxy));
}

// Antisymmetric differences x(c+o) - x(c-o) over the 7 Kuhn directions.
template <class T>
struct Diff7 {
  T e1, e2, e3, f12, f23, f13, b;
};

template <class T, class V>
__device__ __forceinline__ Diff7<T> diff7v(const V& x) {
  Diff7<T> d;
  d.e1 = x(1, 0, 0) - x(-1, 0, 0);
  d.e2 = x(0, 1, 0) - x(0, -1, 0);
  d.e3 = x(0, 0, 1) - x(0, 0, -1);
  d.f12 = x(1, 1, 0) - x(-1, -1, 0);
  d.f23 = x(0, 1, 1) - x(0, -1, -1);
  d.f13 = x(1, 0, 1) - x(-1, 0, -1);
  d.b = x(1, 1, 1) - x(-1, -1, -1);
  return d;
}

template <class T>
__device__ __forceinline__ Diff7<T> diff7(const T* x, const Node& n, int64_t px, int64_t pxy) {
  return diff7v<T>(gnb(x, n, px, pxy));
}

// 12 * Div_d from the differences.
template <class T>
__device__ __forceinline__ void div12_all(const Diff7<T>& d, T out[3]) {
  const T s = ((d.e1 + d.e2) + (d.e3 + d.f12)) + ((d.f23 + d.f13) - d.b);
  out[0] = s - (T)2 * (d.f12 + d.f13) - (T)4 * d.e1;
  out[1] = s - (T)2 * (d.f12 + d.f23) - (T)4 * d.e2;
  out[2] = s - (T)2 * (d.f13 + d.f23) - (T)4 * d.e3;
}

template <class T>
__device__ __forceinline__ T div12(const Diff7<T>& d, int comp) {
  const T s = ((d.e1 + d.e2) + (d.e3 + d.f12)) + ((d.f23 + d.f13) - d.b);
  if (comp == 0) return s - (T)2 * (d.f12 + d.f13) - (T)4 * d.e1;
  if (comp == 1) return s - (T)2 * (d.f12 + d.f23) - (T)4 * d.e2;
  return s - (T)2 * (d.f13 + d.f23) - (T)4 * d.e3;
}

// --- rows of boundary nodes from the class table ------------------------------
// Table layout per class (unit lattice spacing): [W_LAP,+15) stiffness row,
// [W_B+15d,+15) B_d row, [W_BT+15d,+15) B_d^T row, [W_M,+15) mass row,
// [W_LUMP] lumped mass.  Offsets: 0 centre, 1..7 = +o, 8..14 = -o over the
// Kuhn directions e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3.

// Off-centre part sum_{o=1..14} w[o] x(c+o), in offset order.
template <class T, class V>
__device__ __forceinline__ T st14v(const V& x, const T* w, T acc) {
  acc += w[1] * x(1, 0, 0);
  acc += w[2] * x(0, 1, 0);
  acc += w[3] * x(0, 0, 1);
  acc += w[4] * x(1, 1, 0);
  acc += w[5] * x(0, 1, 1);
  acc += w[6] * x(1, 0, 1);
  acc += w[7] * x(1, 1, 1);
  acc += w[8] * x(-1, 0, 0);
  acc += w[9] * x(0, -1, 0);
  acc += w[10] * x(0, 0, -1);
  acc += w[11] * x(-1, -1, 0);
  acc += w[12] * x(0, -1, -1);
  acc += w[13] * x(-1, 0, -1);
  acc += w[14] * x(-1, -1, -1);
  return acc;
}

template <class T, class V>
__device__ __forceinline__ T st15v(const V& x, const T* w) {
  return st14v<T>(x, w, w[0] * x(0, 0, 0));
}

template <class T>
__device__ __forceinline__ const T* class_row(const LevelDev<T>& L, int64_t c) {
  return L.wt + (int64_t)W_STRIDE * L.cls[c];
}

// Unit stiffness row split into diagonal and off-diagonal sum (Gauss-Seidel).
template <class T, class V>
__device__ __forceinline__ void irr_lap_parts_v(const V& x, const T* w, T& dg, T& of) {
  dg = w[W_LAP];
  of = st14v<T>(x, w + W_LAP, (T)0);
}

template <class T>
__device__ __forceinline__ void irr_lap_parts(const LevelDev<T>& L, const T* x, const Node& n, T& dg, T& of) {
  irr_lap_parts_v<T>(gnb(x, n, L.px, L.pxy), class_row(L, n.c), dg, of);
}

// Consistent mass row (times h^3).
template <class T>
__device__ __forceinline__ T irr_mass_row(const LevelDev<T>& L, const T* x, const Node& n) {
  return L.h3 * st15v<T>(gnb(x, n, L.px, L.pxy), class_row(L, n.c) + W_M);
}

// B_d row applied to one scalar field for the three d (times h^2).
template <class T>
__device__ __forceinline__ void irr_B_scalar(const LevelDev<T>& L, const T* x, const Node& n, T out[3]) {
  const T* w = class_row(L, n.c);
  const GNb<T> v = gnb(x, n, L.px, L.pxy);
#pragma unroll
  for (int d = 0; d < 3; ++d) out[d] = L.h2 * st15v<T>(v, w + W_B + 15 * d);
}

// --- D form (a_2): the coupled velocity block from its class rows ------------

template <class T>
__device__ __forceinline__ const T* d_row(const LevelDev<T>& L, int64_t c) {
  return L.wt2 + (int64_t)W2_STRIDE * L.cls[c];
}

// (A2 u)_a at the node for a = 0, 1, 2 (times nu h).
template <class T, class V>
__device__ __forceinline__ void row_A2_v(const LevelDev<T>& L, const V* u, const T* w2, T out[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out[a] = L.nuh * ((st15v<T>(u[0], w2 + 15 * (3 * a)) + st15v<T>(u[1], w2 + 15 * (3 * a + 1))) +
                      st15v<T>(u[2], w2 + 15 * (3 * a + 2)));
}

// Node-block Gauss-Seidel update: the node's three components solve
// D (u_new) = r - (off-centre part of A2 u), D the 3 x 3 centre block.
template <class T, class V>
__device__ __forceinline__ void vel_block_value(const LevelDev<T>& L, const T* w2, const T r[3], const V* u,
                                                T out[3]) {
  T s[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    s[a] = r[a] - L.nuh * ((st14v<T>(u[0], w2 + 15 * (3 * a), (T)0) + st14v<T>(u[1], w2 + 15 * (3 * a + 1), (T)0)) +
                           st14v<T>(u[2], w2 + 15 * (3 * a + 2), (T)0));
  const T* di = w2 + W2_DINV;
  const T inv = (T)1 / L.nuh;
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = inv * ((di[3 * a] * s[0] + di[3 * a + 1] * s[1]) + di[3 * a + 2] * s[2]);
}

// --- full rows of the Stokes operator ----------------------------------------
// View forms take the class row w of the node (used when fl has F_IRR).

// (A u_d)_node for all d (nodes with F_VFREE).
template <class T, class V>
__device__ __forceinline__ void row_A_v(const LevelDev<T>& L, const V* u, const T* w, uint8_t fl, T out[3]) {
  if (!(fl & F_IRR)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = L.nuh * ((T)6 * u[d](0, 0, 0) - nb6v(u[d]));
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = L.nuh * st15v<T>(u[d], w + W_LAP);
  }
}

// (B_d^T p)_node for all d.
template <class T, class V>
__device__ __forceinline__ void row_BT_v(const LevelDev<T>& L, const V& p, const T* w, uint8_t fl, T out[3]) {
  if (!(fl & F_IRR)) {
    const Diff7<T> dp = diff7v<T>(p);
    T dv[3];
    div12_all(dp, dv);
    const T s = -L.h2 * (T)(1.0 / 12.0);
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = s * dv[d];
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = L.h2 * st15v<T>(p, w + W_BT + 15 * d);
  }
}

// (sum_d B_d u_d)_node.
template <class T, class V>
__device__ __forceinline__ T row_B_v(const LevelDev<T>& L, const V* u, const T* w, uint8_t fl) {
  if (!(fl & F_IRR)) {
    const T d0 = div12(diff7v<T>(u[0]), 0);
    const T d1 = div12(diff7v<T>(u[1]), 1);
    const T d2 = div12(diff7v<T>(u[2]), 2);
    return L.h2 * (T)(1.0 / 12.0) * ((d0 + d1) + d2);
  }
  return L.h2 * ((st15v<T>(u[0], w + W_B) + st15v<T>(u[1], w + W_B + 15)) + st15v<T>(u[2], w + W_B + 30));
}

// (C p)_node.
template <class T, class V>
__device__ __forceinline__ T row_C_v(const LevelDev<T>& L, const V& p, const T* w, uint8_t fl) {
  if (!(fl & F_IRR)) return L.c * ((T)6 * p(0, 0, 0) - nb6v(p));
  return L.c * st15v<T>(p, w + W_LAP);
}

// Pointer forms over the padded global arrays.
template <class T>
__device__ __forceinline__ const T* row_of(const LevelDev<T>& L, int64_t c, uint8_t fl) {
  return (fl & F_IRR) ? class_row(L, c) : nullptr;
}

template <class T>
__device__ __forceinline__ void row_A(const LevelDev<T>& L, const T* const* u, const Node& n, uint8_t fl, T out[3]) {
  const GNb<T> v[3] = {gnb(u[0], n, L.px, L.pxy), gnb(u[1], n, L.px, L.pxy), gnb(u[2], n, L.px, L.pxy)};
  if (L.wt2)
    row_A2_v(L, v, d_row(L, n.c), out);
  else
    row_A_v(L, v, row_of(L, n.c, fl), fl, out);
}

template <class T>
__device__ __forceinline__ void row_BT(const LevelDev<T>& L, const T* p, const Node& n, uint8_t fl, T out[3]) {
  row_BT_v(L, gnb(p, n, L.px, L.pxy), row_of(L, n.c, fl), fl, out);
}

template <class T>
__device__ __forceinline__ T row_B(const LevelDev<T>& L, const T* const* u, const Node& n, uint8_t fl) {
  const GNb<T> v[3] = {gnb(u[0], n, L.px, L.pxy), gnb(u[1], n, L.px, L.pxy), gnb(u[2], n, L.px, L.pxy)};
  return row_B_v(L, v, row_of(L, n.c, fl), fl);
}

template <class T>
__device__ __forceinline__ T row_C(const LevelDev<T>& L, const T* p, const Node& n, uint8_t fl) {
  return row_C_v(L, gnb(p, n, L.px, L.pxy), row_of(L, n.c, fl), fl);
}

// Free slip (Sec. 6.1): the admissible part of a velocity value or residual
// at a node whose class row w is a free-slip class: v - n (n . v) in the
// tangent plane of the normal n, or t (t . v) along the edge direction t.
template <class T>
__device__ __forceinline__ void slip_project(const T* w, T v[3]) {
  const T kind = w[W_SLIP];
  if (kind != (T)0) {
    const T s = (w[W_NRM] * v[0] + w[W_NRM + 1] * v[1]) + w[W_NRM + 2] * v[2];
    if (kind == (T)1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] -= s * w[W_NRM + d];
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] = s * w[W_NRM + d];
    }
  }
}

// Lumped pressure mass m_i = int phi_i.
template <class T>
__device__ __forceinline__ T lumped_mass(const LevelDev<T>& L, int64_t c, uint8_t fl) {
  if (!(fl & F_IRR)) return L.h3;
  return L.h3 * class_row(L, c)[W_LUMP];
}

}  // namespace hhg
