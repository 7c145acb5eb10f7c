// Device-side level views and stencil arithmetic of the P1-P1 Stokes operator
// on the Kuhn lattice.
//
// Storage: every field of a level is one padded 3-D array over the lattice
// with a zero ghost frame of one node, x fastest: node (i,j,k) lives at
// (i+1) + px (j+1) + pxy (k+1).  Fields are zero on nodes without the
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
// tetrahedra active).  Nodes flagged F_IRR instead sum the element matrices
// of their active incident tetrahedra (for_incident below), which is the
// plain definition of the assembled row.
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
  T nuh;                 // nu * h
  T c;                   // delta * h_T^2 * h
  T h2;                  // h^2
  T h3;                  // h^3
  T dh2;                 // delta * h_T^2
  T omega;               // pressure under-relaxation
  T* u[3];
  T* p;
  T* f[3];
  T* g;
  T* r[3];
  T* rp;
};

__device__ __forceinline__ int64_t pidx(int64_t px, int64_t pxy, int i, int j, int k) {
  return (int64_t)(i + 1) + px * (j + 1) + pxy * (k + 1);
}

template <class T>
__device__ __forceinline__ T nb6(const T* __restrict__ x, int64_t c, int64_t px, int64_t pxy) {
  return ((x[c - 1] + x[c + 1]) + (x[c - px] + x[c + px])) + (x[c - pxy] + x[c + pxy]);
}

// Antisymmetric differences x(c+o) - x(c-o) over the 7 Kuhn directions.
template <class T>
struct Diff7 {
  T e1, e2, e3, f12, f23, f13, b;
};

template <class T>
__device__ __forceinline__ Diff7<T> diff7(const T* __restrict__ x, int64_t c, int64_t px, int64_t pxy) {
  Diff7<T> d;
  d.e1 = x[c + 1] - x[c - 1];
  d.e2 = x[c + px] - x[c - px];
  d.e3 = x[c + pxy] - x[c - pxy];
  d.f12 = x[c + 1 + px] - x[c - 1 - px];
  d.f23 = x[c + px + pxy] - x[c - px - pxy];
  d.f13 = x[c + 1 + pxy] - x[c - 1 - pxy];
  d.b = x[c + 1 + px + pxy] - x[c - 1 - px - pxy];
  return d;
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

// Visit the active tetrahedra incident to node (i,j,k): fn(m, s, v) with m
// the node's local vertex number along path s and v[4] the padded indices
// of the tetrahedron's vertices in path order.
template <class T, class F>
__device__ __forceinline__ void for_incident(const LevelDev<T>& L, int i, int j, int k, F&& fn) {
  const int64_t step[3] = {1, L.px, L.pxy};
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    const int cx = i - qx, cy = j - qy, cz = k - qz;
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      const int m = corner_local(s, qx, qy, qz);
      if (m < 0) continue;
      if (!tet_active(L.mmask, L.mx, L.my, L.mz, L.level, cx, cy, cz, s)) continue;
      int64_t v[4];
      v[0] = pidx(L.px, L.pxy, cx, cy, cz);
      v[1] = v[0] + step[path_axis(s, 0)];
      v[2] = v[1] + step[path_axis(s, 1)];
      v[3] = v[0] + 1 + L.px + L.pxy;
      fn(m, s, v);
    }
  }
}

// --- element-sum rows for irregular nodes ---------------------------------

// Row of the unit stiffness sum: diag = sum_T K6[m][m] / 6, off = sum_T sum_{n != m} K6[m][n] x_n / 6.
template <class T>
__device__ __forceinline__ void irr_lap_row(const LevelDev<T>& L, const T* x, int i, int j, int k,
                                            T& diag, T& off) {
  T dg = 0, of = 0;
  for_incident(L, i, j, k, [&](int m, int, const int64_t* v) {
    dg += (T)kuhn_stiff6(m, m);
    if (m > 0) of -= x[v[m - 1]];
    if (m < 3) of -= x[v[m + 1]];
  });
  diag = dg * (T)(1.0 / 6.0);
  off = of * (T)(1.0 / 6.0);
}

// (Lap x)_node as an element sum (unit scale).
template <class T>
__device__ __forceinline__ T irr_lap(const LevelDev<T>& L, const T* x, int i, int j, int k, int64_t c) {
  T dg, of;
  irr_lap_row(L, x, i, j, k, dg, of);
  return dg * x[c] + of;
}

// 24 * (B_d x)_node / (-h^2) summed over elements: sum_T (x_{s+1} - x_s) along
// the path step s whose axis is d.  Returns the three components.
template <class T>
__device__ __forceinline__ void irr_grad_sum(const LevelDev<T>& L, const T* const* x3, int i, int j, int k,
                                             T out[3]) {
  out[0] = out[1] = out[2] = 0;
  for_incident(L, i, j, k, [&](int, int s, const int64_t* v) {
#pragma unroll
    for (int st = 0; st < 3; ++st) {
      const int d = path_axis(s, st);
      out[d] += x3[d][v[st + 1]] - x3[d][v[st]];
    }
  });
}

// Same for a single scalar field applied to all three directions.
template <class T>
__device__ __forceinline__ void irr_grad_scalar(const LevelDev<T>& L, const T* x, int i, int j, int k, T out[3]) {
  out[0] = out[1] = out[2] = 0;
  for_incident(L, i, j, k, [&](int, int s, const int64_t* v) {
#pragma unroll
    for (int st = 0; st < 3; ++st) out[path_axis(s, st)] += x[v[st + 1]] - x[v[st]];
  });
}

// 24 * (B_d^T p)_node / (-h^2) = sum_T g_{m,d} sum_n p_n with the unit
// barycentric gradient g_m = e_{a(m-1)} - e_{a(m)} (a = path axes).
template <class T>
__device__ __forceinline__ void irr_gradT(const LevelDev<T>& L, const T* p, int i, int j, int k, T out[3]) {
  out[0] = out[1] = out[2] = 0;
  for_incident(L, i, j, k, [&](int m, int s, const int64_t* v) {
    const T sum = (p[v[0]] + p[v[1]]) + (p[v[2]] + p[v[3]]);
    if (m >= 1) out[path_axis(s, m - 1)] += sum;
    if (m <= 2) out[path_axis(s, m)] -= sum;
  });
}

// 120/h^3 * (M x)_node = sum_T (x_m + sum_n x_n)
template <class T>
__device__ __forceinline__ T irr_mass(const LevelDev<T>& L, const T* x, int i, int j, int k) {
  T acc = 0;
  for_incident(L, i, j, k, [&](int m, int, const int64_t* v) {
    acc += x[v[m]] + ((x[v[0]] + x[v[1]]) + (x[v[2]] + x[v[3]]));
  });
  return acc;
}

template <class T>
__device__ __forceinline__ int irr_count(const LevelDev<T>& L, int i, int j, int k) {
  int n = 0;
  for_incident(L, i, j, k, [&](int, int, const int64_t*) { ++n; });
  return n;
}

// --- boundary-row paths ------------------------------------------------------
// The element-sum rows run only on nodes flagged F_IRR.  They are kept out of
// line: each gets its own stack frame, the regular fast path of every kernel
// stays small, and no local array of a caller can share storage with the
// temporaries of these loops.

template <class T>
__device__ __noinline__ void irr_row_A(const LevelDev<T>& L, const T* u0, const T* u1, const T* u2, int i, int j,
                                       int k, int64_t c, T* out) {
  out[0] = L.nuh * irr_lap(L, u0, i, j, k, c);
  out[1] = L.nuh * irr_lap(L, u1, i, j, k, c);
  out[2] = L.nuh * irr_lap(L, u2, i, j, k, c);
}

template <class T>
__device__ __noinline__ T irr_row_A1(const LevelDev<T>& L, const T* x, int i, int j, int k, int64_t c) {
  return L.nuh * irr_lap(L, x, i, j, k, c);
}

template <class T>
__device__ __noinline__ void irr_row_BT(const LevelDev<T>& L, const T* p, int i, int j, int k, T* out) {
  T gs[3];
  irr_gradT(L, p, i, j, k, gs);
  const T s = -L.h2 * (T)(1.0 / 24.0);
  out[0] = s * gs[0];
  out[1] = s * gs[1];
  out[2] = s * gs[2];
}

template <class T>
__device__ __noinline__ T irr_row_B(const LevelDev<T>& L, const T* u0, const T* u1, const T* u2, int i, int j,
                                    int k) {
  const T* x3[3] = {u0, u1, u2};
  T gs[3];
  irr_grad_sum(L, x3, i, j, k, gs);
  return -L.h2 * (T)(1.0 / 24.0) * ((gs[0] + gs[1]) + gs[2]);
}

template <class T>
__device__ __noinline__ T irr_row_C(const LevelDev<T>& L, const T* p, int i, int j, int k, int64_t c) {
  return L.c * irr_lap(L, p, i, j, k, c);
}

// Diagonal and off-diagonal sum of the unit Laplacian row (Gauss-Seidel updates).
template <class T>
__device__ __noinline__ void irr_lap_parts(const LevelDev<T>& L, const T* x, int i, int j, int k, T* dg_of) {
  T dg, of;
  irr_lap_row(L, x, i, j, k, dg, of);
  dg_of[0] = dg;
  dg_of[1] = of;
}

template <class T>
__device__ __noinline__ T irr_mass_row(const LevelDev<T>& L, const T* x, int i, int j, int k) {
  return L.h3 * (T)(1.0 / 120.0) * irr_mass(L, x, i, j, k);
}

template <class T>
__device__ __noinline__ void irr_grad_scalar_row(const LevelDev<T>& L, const T* x, int i, int j, int k, T* out) {
  T gs[3];
  irr_grad_scalar(L, x, i, j, k, gs);
  const T s = -L.h2 * (T)(1.0 / 24.0);
  out[0] = s * gs[0];
  out[1] = s * gs[1];
  out[2] = s * gs[2];
}

template <class T>
__device__ __noinline__ T irr_lumped(const LevelDev<T>& L, int i, int j, int k) {
  return L.h3 * (T)(1.0 / 24.0) * (T)irr_count(L, i, j, k);
}

// --- full rows of the Stokes operator ----------------------------------------

// (A u_d)_node for all d (nodes with F_VFREE).
template <class T>
__device__ __forceinline__ void row_A(const LevelDev<T>& L, const T* const* u, int i, int j, int k, int64_t c,
                                      uint8_t fl, T out[3]) {
  if (!(fl & F_IRR)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = L.nuh * ((T)6 * u[d][c] - nb6(u[d], c, L.px, L.pxy));
  } else {
    irr_row_A(L, u[0], u[1], u[2], i, j, k, c, out);
  }
}

// (B_d^T p)_node for all d.
template <class T>
__device__ __forceinline__ void row_BT(const LevelDev<T>& L, const T* p, int i, int j, int k, int64_t c, uint8_t fl,
                                       T out[3]) {
  if (!(fl & F_IRR)) {
    const Diff7<T> dp = diff7(p, c, L.px, L.pxy);
    T dv[3];
    div12_all(dp, dv);
    const T s = -L.h2 * (T)(1.0 / 12.0);
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = s * dv[d];
  } else {
    irr_row_BT(L, p, i, j, k, out);
  }
}

// (sum_d B_d u_d)_node.
template <class T>
__device__ __forceinline__ T row_B(const LevelDev<T>& L, const T* const* u, int i, int j, int k, int64_t c,
                                   uint8_t fl) {
  if (!(fl & F_IRR)) {
    const T d0 = div12(diff7(u[0], c, L.px, L.pxy), 0);
    const T d1 = div12(diff7(u[1], c, L.px, L.pxy), 1);
    const T d2 = div12(diff7(u[2], c, L.px, L.pxy), 2);
    return L.h2 * (T)(1.0 / 12.0) * ((d0 + d1) + d2);
  }
  return irr_row_B(L, u[0], u[1], u[2], i, j, k);
}

// (C p)_node.
template <class T>
__device__ __forceinline__ T row_C(const LevelDev<T>& L, const T* p, int i, int j, int k, int64_t c, uint8_t fl) {
  if (!(fl & F_IRR)) return L.c * ((T)6 * p[c] - nb6(p, c, L.px, L.pxy));
  return irr_row_C(L, p, i, j, k, c);
}

// Lumped pressure mass m_i = int phi_i.
template <class T>
__device__ __forceinline__ T lumped_mass(const LevelDev<T>& L, int i, int j, int k, uint8_t fl) {
  if (!(fl & F_IRR)) return L.h3;
  return irr_lumped(L, i, j, k);
}

}  // namespace hhg
