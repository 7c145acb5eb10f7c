// Per-node bodies of the smoother, residual and transfer steps (Sec. 3.3-3.5).
// The grid kernels run one node per thread; the fused coarse-levels kernel
// loops over the nodes of a level inside one thread block.  Both call these
// functions, so the two paths do the same arithmetic in the same order.
#pragma once
#include "hhg_device.cuh"

namespace hhg {

// Velocity block of the level: DF = 1 the D form (coupled 3 x 3 node blocks),
// 0 the Laplace form, -1 read from the level (L.wt2 set in the D form).  The
// grid kernels are instantiated per form, so that a kernel of one form does
// not carry the other form's registers.
template <int DF, class T>
__device__ __forceinline__ bool d_form(const LevelDev<T>& L) {
  return DF < 0 ? L.wt2 != nullptr : DF == 1;
}

// RU = F - B^T P (velocity nodes).
template <class T>
__device__ __forceinline__ void node_vel_rhs(const LevelDev<T>& L, const Node& n) {
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  if (!(fl & F_VFREE)) return;
  T bt[3];
  row_BT(L, L.p, n, fl, bt);
#pragma unroll
  for (int d = 0; d < 3; ++d) L.r[d][c] = L.f[d][c] - bt[d];
}

// The colour updates come in two forms.  SPEC (for small, latency-bound
// levels) evaluates the regular-node (closed-form stencil) update before it
// reads the node's flags, so that its loads are not gated by the flag load;
// a boundary node then recomputes with its class rows, and a node without
// the unknown stores nothing.  The other form (for large, throughput-bound
// levels, where the speculative loads and arithmetic of boundary and
// Dirichlet nodes cost more than the latency they hide) reads the flags
// first.  Both store the same values.  u, p are neighbour views centred on
// the node (global arrays, a shared-memory tile, or plane-pointer tables).

// u_d <- u_d + (RU_d - (A u_d)) / A_ii  (one node of the current colour);
// in the D form the node's three components at once with its 3 x 3 block.
template <bool SPEC, class T, class V, int DF = -1>
__device__ __forceinline__ void node_vel_gs_v(const LevelDev<T>& L, int64_t c, const V* u, T inv6nuh) {
  if (d_form<DF>(L)) {
    if (!(L.flags[c] & F_VFREE)) return;
    const T r[3] = {L.r[0][c], L.r[1][c], L.r[2][c]};
    T out[3];
    vel_block_value(L, d_row(L, c), r, u, out);
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][c] = out[d];
    return;
  }
  T reg[3];
  uint8_t fl;
  if (SPEC) {
#pragma unroll
    for (int d = 0; d < 3; ++d) reg[d] = (L.r[d][c] + L.nuh * nb6v(u[d])) * inv6nuh;
    fl = L.flags[c];
    if (!(fl & F_VFREE)) return;
  } else {
    fl = L.flags[c];
    if (!(fl & F_VFREE)) return;
    if (!(fl & F_IRR)) {
#pragma unroll
      for (int d = 0; d < 3; ++d) reg[d] = (L.r[d][c] + L.nuh * nb6v(u[d])) * inv6nuh;
    }
  }
  if (!(fl & F_IRR)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][c] = reg[d];
    return;
  }
  const T* w = class_row(L, c);
  T out[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T dg, of;
    irr_lap_parts_v<T>(u[d], w, dg, of);
    out[d] = (L.r[d][c] - L.nuh * of) / (L.nuh * dg);
  }
  slip_project(w, out);
#pragma unroll
  for (int d = 0; d < 3; ++d) L.u[d][c] = out[d];
}

template <bool SPEC, class T, int DF = -1>
__device__ __forceinline__ void node_vel_gs(const LevelDev<T>& L, const Node& n, T inv6nuh) {
  const GNb<T> u[3] = {gnb(L.u[0], n, L.px, L.pxy), gnb(L.u[1], n, L.px, L.pxy), gnb(L.u[2], n, L.px, L.pxy)};
  node_vel_gs_v<SPEC, T, GNb<T>, DF>(L, n.c, u, inv6nuh);
}

// New velocity of a regular node from its right-hand side f (3 values) and
// f - B^T p formed at the node: the node's own old value does not enter.
template <class T, class V>
__device__ __forceinline__ void vel_regular_value(const LevelDev<T>& L, const T* f, const V* u, const V& p,
                                                  T inv6nuh, T reg[3]) {
  T dv[3];
  div12_all(diff7v<T>(p), dv);
  const T s = -L.h2 * (T)(1.0 / 12.0);
#pragma unroll
  for (int d = 0; d < 3; ++d) reg[d] = ((f[d] - s * dv[d]) + L.nuh * nb6v(u[d])) * inv6nuh;
}

// New velocity of a boundary node from its class row w.
template <class T, class V>
__device__ __forceinline__ void vel_irr_value(const LevelDev<T>& L, const T* w, const T* f, const V* u, const V& p,
                                              T out[3]) {
  T bt[3];
  row_BT_v(L, p, w, F_IRR, bt);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T dg, of;
    irr_lap_parts_v<T>(u[d], w, dg, of);
    out[d] = ((f[d] - bt[d]) - L.nuh * of) / (L.nuh * dg);
  }
  slip_project(w, out);
}

// Regular-node velocity update with f - B^T p formed at the node.  The same
// arithmetic as vel_regular_value, with f read where it is used: loading it
// ahead of the stencil keeps three more values live across the neighbour
// loads and costs the grid kernels a resident block per SM.
template <class T, class V>
__device__ __forceinline__ void vel_rhs_regular(const LevelDev<T>& L, int64_t c, const V* u, const V& p, T inv6nuh,
                                                T reg[3]) {
  T dv[3];
  div12_all(diff7v<T>(p), dv);
  const T s = -L.h2 * (T)(1.0 / 12.0);
#pragma unroll
  for (int d = 0; d < 3; ++d) reg[d] = ((L.f[d][c] - s * dv[d]) + L.nuh * nb6v(u[d])) * inv6nuh;
}

// Velocity update of a boundary node (class rows) with f - B^T p formed at
// the node (the arithmetic of vel_irr_value).
template <class T, class V>
__device__ __forceinline__ void vel_rhs_irr(const LevelDev<T>& L, int64_t c, const V* u, const V& p) {
  const T* w = class_row(L, c);
  T bt[3], out[3];
  row_BT_v(L, p, w, F_IRR, bt);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T dg, of;
    irr_lap_parts_v<T>(u[d], w, dg, of);
    out[d] = ((L.f[d][c] - bt[d]) - L.nuh * of) / (L.nuh * dg);
  }
  slip_project(w, out);
#pragma unroll
  for (int d = 0; d < 3; ++d) L.u[d][c] = out[d];
}

// Same update with the right-hand side f - B^T p formed at the node (p does
// not change during the velocity sweeps, Sec. 3.3), RU is not touched.
template <bool SPEC, class T, class V, int DF = -1>
__device__ __forceinline__ void node_vel_gs_rhs_v(const LevelDev<T>& L, int64_t c, const V* u, const V& p,
                                                  T inv6nuh) {
  if (d_form<DF>(L)) {
    const uint8_t fl = L.flags[c];
    if (!(fl & F_VFREE)) return;
    T bt[3];
    row_BT_v(L, p, row_of(L, c, fl), fl, bt);
    const T r[3] = {L.f[0][c] - bt[0], L.f[1][c] - bt[1], L.f[2][c] - bt[2]};
    T out[3];
    vel_block_value(L, d_row(L, c), r, u, out);
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][c] = out[d];
    return;
  }
  T reg[3];
  uint8_t fl;
  if (SPEC) {
    vel_rhs_regular(L, c, u, p, inv6nuh, reg);
    fl = L.flags[c];
    if (!(fl & F_VFREE)) return;
  } else {
    fl = L.flags[c];
    if (!(fl & F_VFREE)) return;
    if (!(fl & F_IRR)) vel_rhs_regular(L, c, u, p, inv6nuh, reg);
  }
  if (!(fl & F_IRR)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][c] = reg[d];
    return;
  }
  vel_rhs_irr(L, c, u, p);
}

template <bool SPEC, class T, int DF = -1>
__device__ __forceinline__ void node_vel_gs_rhs(const LevelDev<T>& L, const Node& n, T inv6nuh) {
  const GNb<T> u[3] = {gnb(L.u[0], n, L.px, L.pxy), gnb(L.u[1], n, L.px, L.pxy), gnb(L.u[2], n, L.px, L.pxy)};
  node_vel_gs_rhs_v<SPEC, T, GNb<T>, DF>(L, n.c, u, gnb(L.p, n, L.px, L.pxy), inv6nuh);
}

// RP = B U - G (pressure nodes).
template <class T>
__device__ __forceinline__ void node_pres_rhs(const LevelDev<T>& L, const Node& n) {
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  if (!(fl & F_ACT)) return;
  const T* uu[3] = {L.u[0], L.u[1], L.u[2]};
  L.rp[c] = row_B(L, uu, n, fl) - L.g[c];
}

// p <- p + omega (RP - C p) / C_ii  (forward SOR sweep from zero, Sec. 3.5).
template <class T>
__device__ __forceinline__ void node_pres_gs(const LevelDev<T>& L, const Node& n, T omega_over_6c) {
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  if (!(fl & F_ACT)) return;
  const T pc = L.p[c];
  if (!(fl & F_IRR)) {
    const T cp = L.c * ((T)6 * pc - nb6(L.p, n, L.px, L.pxy));
    L.p[c] = pc + omega_over_6c * (L.rp[c] - cp);
  } else {
    T dg, of;
    irr_lap_parts(L, L.p, n, dg, of);
    const T cp = L.c * (dg * pc + of);
    L.p[c] = pc + L.omega * (L.rp[c] - cp) / (L.c * dg);
  }
}

// New pressure of a regular node from its right-hand side g, B u - g formed at
// the node, and its old value pc.
template <class T, class V>
__device__ __forceinline__ T pres_regular_value(const LevelDev<T>& L, T g, const V* u, const V& p, T pc,
                                                T omega_over_6c) {
  const T d0 = div12(diff7v<T>(u[0]), 0);
  const T d1 = div12(diff7v<T>(u[1]), 1);
  const T d2 = div12(diff7v<T>(u[2]), 2);
  const T rp = L.h2 * (T)(1.0 / 12.0) * ((d0 + d1) + d2) - g;
  const T cp = L.c * ((T)6 * pc - nb6v(p));
  return pc + omega_over_6c * (rp - cp);
}

// New pressure of a boundary node from its class row w.
template <class T, class V>
__device__ __forceinline__ T pres_irr_value(const LevelDev<T>& L, const T* w, T g, const V* u, const V& p, T pc) {
  const T rp = row_B_v(L, u, w, F_IRR) - g;
  T dg, of;
  irr_lap_parts_v<T>(p, w, dg, of);
  const T cp = L.c * (dg * pc + of);
  return pc + L.omega * (rp - cp) / (L.c * dg);
}

// Regular-node pressure update with B u - g formed at the node.
template <class T, class V>
__device__ __forceinline__ T pres_rhs_regular(const LevelDev<T>& L, int64_t c, const V* u, const V& p, T pc,
                                              T omega_over_6c) {
  return pres_regular_value(L, L.g[c], u, p, pc, omega_over_6c);
}

// Pressure update of a boundary node (class rows) with B u - g formed at the node.
template <class T, class V>
__device__ __forceinline__ void pres_rhs_irr(const LevelDev<T>& L, int64_t c, const V* u, const V& p, T pc) {
  L.p[c] = pres_irr_value(L, class_row(L, c), L.g[c], u, p, pc);
}

// Same update with B u - g formed at the node (u does not change during the
// pressure sweep), RP is not touched.
template <bool SPEC, class T, class V>
__device__ __forceinline__ void node_pres_gs_rhs_v(const LevelDev<T>& L, int64_t c, const V* u, const V& p,
                                                   T omega_over_6c) {
  T reg = (T)0, pc;
  uint8_t fl;
  if (SPEC) {
    pc = p(0, 0, 0);
    reg = pres_rhs_regular(L, c, u, p, pc, omega_over_6c);
    fl = L.flags[c];
    if (!(fl & F_ACT)) return;
  } else {
    fl = L.flags[c];
    if (!(fl & F_ACT)) return;
    pc = p(0, 0, 0);
    if (!(fl & F_IRR)) reg = pres_rhs_regular(L, c, u, p, pc, omega_over_6c);
  }
  if (!(fl & F_IRR)) {
    L.p[c] = reg;
    return;
  }
  pres_rhs_irr(L, c, u, p, pc);
}

template <bool SPEC, class T>
__device__ __forceinline__ void node_pres_gs_rhs(const LevelDev<T>& L, const Node& n, T omega_over_6c) {
  const GNb<T> u[3] = {gnb(L.u[0], n, L.px, L.pxy), gnb(L.u[1], n, L.px, L.pxy), gnb(L.u[2], n, L.px, L.pxy)};
  node_pres_gs_rhs_v<SPEC>(L, n.c, u, gnb(L.p, n, L.px, L.pxy), omega_over_6c);
}

// (RU, RP) = (F, G) - K (U, P) at one node, returned in r[0..3]; zero for
// unknowns the node does not carry.
template <class T, class V, int DF = -1>
__device__ __forceinline__ void node_residual_v(const LevelDev<T>& L, int64_t c, uint8_t fl, const V* u, const V& p,
                                                T r[4]) {
  const T* w = row_of(L, c, fl);
  if (fl & F_VFREE) {
    T au[3], bt[3];
    if (d_form<DF>(L))
      row_A2_v(L, u, d_row(L, c), au);
    else
      row_A_v(L, u, w, fl, au);
    row_BT_v(L, p, w, fl, bt);
#pragma unroll
    for (int d = 0; d < 3; ++d) r[d] = L.f[d][c] - au[d] - bt[d];
    if (fl & F_SLIP) slip_project(w, r);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) r[d] = (T)0;
  }
  r[3] = (fl & F_ACT) ? L.g[c] - row_B_v(L, u, w, fl) + row_C_v(L, p, w, fl) : (T)0;
}

template <class T, int DF = -1>
__device__ __forceinline__ void node_residual(const LevelDev<T>& L, const Node& n) {
  const int64_t c = n.c;
  const uint8_t fl = L.flags[c];
  const GNb<T> u[3] = {gnb(L.u[0], n, L.px, L.pxy), gnb(L.u[1], n, L.px, L.pxy), gnb(L.u[2], n, L.px, L.pxy)};
  T r[4];
  node_residual_v<T, GNb<T>, DF>(L, c, fl, u, gnb(L.p, n, L.px, L.pxy), r);
#pragma unroll
  for (int d = 0; d < 3; ++d) L.r[d][c] = r[d];
  L.rp[c] = r[3];
}

// Coarse (F, G) at coarse node (i,j,k) = P^T (RU, RP): P1 interpolation is
// the identity on coarse nodes and the mean of the two ends on coarse-edge
// midpoints, which on the Kuhn lattice are the 14 neighbours along the Kuhn
// directions.  The coarse iterate (U, P) starts from zero.
template <class T>
__device__ __forceinline__ void node_restrict(const LevelDev<T>& Lf, const LevelDev<T>& Lc, int i, int j, int k) {
  const int64_t cc = pidx(Lc.px, Lc.pxy, i, j, k);
  const uint8_t fl = Lc.flags[cc];
  const Node nf = node_at(Lf.px, Lf.pxy, 2 * i, 2 * j, 2 * k);
  T s[4];
  const T* src[4] = {Lf.r[0], Lf.r[1], Lf.r[2], Lf.rp};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const GNb<T> x = gnb(src[q], nf, Lf.px, Lf.pxy);
    // the 14 Kuhn neighbours: +-(e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3)
    T acc = 0;
    acc += x(1, 0, 0) + x(-1, 0, 0);
    acc += x(0, 1, 0) + x(0, -1, 0);
    acc += x(0, 0, 1) + x(0, 0, -1);
    acc += x(1, 1, 0) + x(-1, -1, 0);
    acc += x(0, 1, 1) + x(0, -1, -1);
    acc += x(1, 0, 1) + x(-1, 0, -1);
    acc += x(1, 1, 1) + x(-1, -1, -1);
    s[q] = x(0, 0, 0) + (T)0.5 * acc;
  }
  const bool vf = fl & F_VFREE, ac = fl & F_ACT;
  if (fl & F_SLIP) slip_project(class_row(Lc, cc), s);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Lc.f[d][cc] = vf ? s[d] : (T)0;
    Lc.u[d][cc] = (T)0;
  }
  Lc.g[cc] = ac ? s[3] : (T)0;
  Lc.p[cc] = (T)0;
}

// Fine (U, P) += P (coarse U, P) at fine node (i,j,k).
template <class T>
__device__ __forceinline__ void node_prolong_add(const LevelDev<T>& Lf, const LevelDev<T>& Lc, int i, int j, int k) {
  const int64_t cf = pidx(Lf.px, Lf.pxy, i, j, k);
  const uint8_t fl = Lf.flags[cf];
  if (!(fl & F_ACT)) return;
  const int a = i & 1, b = j & 1, e = k & 1;
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int64_t c0 = pidx(Lc.px, Lc.pxy, I, J, K);
  const bool mid = (a | b | e) != 0;
  const int64_t c1 = pidx(Lc.px, Lc.pxy, I + a, J + b, K + e);
  if (fl & F_VFREE) {
    T v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* x = Lc.u[d];
      v[d] = mid ? (T)0.5 * (x[c0] + x[c1]) : x[c0];
    }
    if (fl & F_SLIP) slip_project(class_row(Lf, cf), v);
#pragma unroll
    for (int d = 0; d < 3; ++d) Lf.u[d][cf] += v[d];
  }
  const T v = mid ? (T)0.5 * (Lc.p[c0] + Lc.p[c1]) : Lc.p[c0];
  Lf.p[cf] += v;
}

}  // namespace hhg
