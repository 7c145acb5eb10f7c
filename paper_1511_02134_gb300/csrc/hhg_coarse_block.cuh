// Coarse-grid solver of the all-at-once multigrid (Sec. 3.7) as a routine of
// one team (a thread-block cluster, or one block; hhg_team.cuh): MINRES on the
// full saddle-point system, preconditioned block-diagonally (Sec. 3.2) with a
// CG solve on each velocity block of A and the inverse lumped pressure mass.
// Always FP64.  Loops have fixed upper trip counts (max iterations).  Used by
// the coarse-solve kernel and by the fused coarse-levels cycle.
//
// Recurrences (start from zero):
//   CG:     stop before an iteration when r.r <= rtol^2 r0.r0 (or r.r = 0),
//           or when d.Ad = 0; at most cg_max iterations.
//   MINRES: Lanczos with Givens rotations; z_j <- z_j / gamma_j,
//           delta_j = (K z_j).z_j, v_{j+1} = K z_j - delta_j/gamma_j v_j
//           - gamma_j/gamma_{j-1} v_{j-1}, z_{j+1} = P^{-1} v_{j+1},
//           gamma_{j+1} = sqrt(z_{j+1}.v_{j+1}); rotation a0..a3, c, s;
//           w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j)/a1; x += c_{j+1} eta w_{j+1};
//           eta <- -s_{j+1} eta; stop when |eta| <= rtol gamma_1.
#pragma once
#include "hhg_kernels.h"
#include "hhg_team.cuh"

namespace hhg {
namespace coarse {


struct V4 {
  double* c[4];
};

struct Ctx {
  LevelDev<double> L;
  Team T;
  int64_t n;  // lattice nodes
};

__device__ __forceinline__ void decode(const LevelDev<double>& L, int64_t q, int& i, int& j, int& k) {
  i = (int)(q % L.nx);
  j = (int)((q / L.nx) % L.ny);
  k = (int)(q / ((int64_t)L.nx * L.ny));
}

__device__ inline double dot4(const Ctx& C, const V4& a, const V4& b) {
  double s = 0;
  for (int64_t q = C.T.rank(); q < C.L.nalloc; q += C.T.size())
    s += (a.c[0][q] * b.c[0][q] + a.c[1][q] * b.c[1][q]) + (a.c[2][q] * b.c[2][q] + a.c[3][q] * b.c[3][q]);
  return team_sum1(C.T, s);
}

// y = K x (zero on entries without unknowns)
__device__ inline void applyK(const Ctx& C, const V4& x, const V4& y) {
  LevelDev<double> L = C.L;
  L.p = x.c[3];
  for (int64_t q = C.T.rank(); q < C.n; q += C.T.size()) {
    int i, j, k;
    decode(L, q, i, j, k);
    const int64_t c = pidx(L.px, L.pxy, i, j, k);
    const uint8_t fl = L.flags[c];
    if (fl & F_VFREE) {
      double au[3], bt[3];
      row_A(L, x.c, c, fl, au);
      row_BT(L, L.p, c, fl, bt);
      for (int d = 0; d < 3; ++d) y.c[d][c] = au[d] + bt[d];
    }
    if (fl & F_ACT) y.c[3][c] = row_B(L, x.c, c, fl) - row_C(L, L.p, c, fl);
  }
  C.T.sync();
}

__device__ __forceinline__ double a_row(const LevelDev<double>& L, const double* x, int64_t c, uint8_t fl) {
  return (fl & F_IRR) ? L.nuh * st15(x, c, offsets15(L.px, L.pxy), class_row(L, c) + W_LAP)
                      : L.nuh * (6.0 * x[c] - nb6(x, c, L.px, L.pxy));
}

// x_d = CG(A, b_d) from zero for the three velocity blocks in lockstep over
// the team: each block follows the stopping rule of cg() on its own (it stops
// before an iteration when r.r <= rtol^2 r0.r0 or r.r = 0, or when d.Ad = 0),
// the others go on; sums of the three blocks share one team reduction.
// f9: 3 scratch fields per block (r, d, A d).  Returns the iterations summed.
__device__ inline int cg3(const Ctx& C, const V4& b, const V4& x, double* const* f9, int max_it, double rtol) {
  const LevelDev<double>& L = C.L;
  for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size()) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x.c[d][q] = 0.0;
      f9[3 * d][q] = b.c[d][q];
      f9[3 * d + 1][q] = b.c[d][q];
      f9[3 * d + 2][q] = 0.0;
    }
  }
  C.T.sync();
  double rr[3] = {0, 0, 0};
  for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size())
#pragma unroll
    for (int d = 0; d < 3; ++d) rr[d] += f9[3 * d][q] * f9[3 * d][q];
  team_sum<3>(C.T, rr);
  double stop[3];
  bool run[3];
  for (int d = 0; d < 3; ++d) {
    stop[d] = rtol * rtol * rr[d];
    run[d] = true;
  }
  int its = 0;
  for (int it = 0; it < max_it; ++it) {
    for (int d = 0; d < 3; ++d)
      if (rr[d] <= stop[d] || rr[d] == 0.0) run[d] = false;
    if (!(run[0] || run[1] || run[2])) break;
    for (int64_t q = C.T.rank(); q < C.n; q += C.T.size()) {
      int i, j, k;
      decode(L, q, i, j, k);
      const int64_t c = pidx(L.px, L.pxy, i, j, k);
      const uint8_t fl = L.flags[c];
      if (!(fl & F_VFREE)) continue;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) f9[3 * d + 2][c] = a_row(L, f9[3 * d + 1], c, fl);
    }
    C.T.sync();
    double dq[3] = {0, 0, 0};
    for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) dq[d] += f9[3 * d + 1][q] * f9[3 * d + 2][q];
    team_sum<3>(C.T, dq);
    double alpha[3];
    for (int d = 0; d < 3; ++d) {
      if (run[d] && dq[d] == 0.0) run[d] = false;
      alpha[d] = run[d] ? rr[d] / dq[d] : 0.0;
    }
    for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) {
          x.c[d][q] += alpha[d] * f9[3 * d + 1][q];
          f9[3 * d][q] -= alpha[d] * f9[3 * d + 2][q];
        }
    C.T.sync();
    double rn[3] = {0, 0, 0};
    for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) rn[d] += f9[3 * d][q] * f9[3 * d][q];
    team_sum<3>(C.T, rn);
    double beta[3];
    for (int d = 0; d < 3; ++d) beta[d] = run[d] ? rn[d] / rr[d] : 0.0;
    for (int64_t q = C.T.rank(); q < L.nalloc; q += C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) f9[3 * d + 1][q] = f9[3 * d][q] + beta[d] * f9[3 * d + 1][q];
    C.T.sync();
    for (int d = 0; d < 3; ++d)
      if (run[d]) {
        rr[d] = rn[d];
        ++its;
      }
  }
  return its;
}

// ---- warp-level CG: the three velocity blocks are solved concurrently ------

// Sum over the warp, the same value in every lane (shuffle tree, lane 0 broadcast).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ inline double wdot(const Ctx& C, const double* a, const double* b) {
  double s = 0;
  for (int64_t q = threadIdx.x & 31; q < C.L.nalloc; q += 32) s += a[q] * b[q];
  return warp_sum(s);
}

__device__ inline void wapplyA(const Ctx& C, const double* x, double* y) {
  const LevelDev<double>& L = C.L;
  for (int64_t q = threadIdx.x & 31; q < C.n; q += 32) {
    int i, j, k;
    decode(L, q, i, j, k);
    const int64_t c = pidx(L.px, L.pxy, i, j, k);
    const uint8_t fl = L.flags[c];
    if (!(fl & F_VFREE)) continue;
    y[c] = (fl & F_IRR) ? L.nuh * st15(x, c, offsets15(L.px, L.pxy), class_row(L, c) + W_LAP)
                        : L.nuh * (6.0 * x[c] - nb6(x, c, L.px, L.pxy));
  }
  __syncwarp();
}

// x = CG(A, b) from zero by one warp (same stopping rule as cg()).
__device__ inline int cg_warp(const Ctx& C, const double* b, double* x, double* r, double* d, double* w, int max_it,
                              double rtol) {
  for (int64_t q = threadIdx.x & 31; q < C.L.nalloc; q += 32) {
    x[q] = 0.0;
    r[q] = b[q];
    d[q] = b[q];
    w[q] = 0.0;
  }
  __syncwarp();
  double rr = wdot(C, r, r);
  const double stop = rtol * rtol * rr;
  int it = 0;
  for (; it < max_it; ++it) {
    if (rr <= stop || rr == 0.0) break;
    wapplyA(C, d, w);
    const double dq = wdot(C, d, w);
    if (dq == 0.0) break;
    const double alpha = rr / dq;
    for (int64_t q = threadIdx.x & 31; q < C.L.nalloc; q += 32) {
      x[q] += alpha * d[q];
      r[q] -= alpha * w[q];
    }
    __syncwarp();
    const double rr_new = wdot(C, r, r);
    const double beta = rr_new / rr;
    for (int64_t q = threadIdx.x & 31; q < C.L.nalloc; q += 32) d[q] = r[q] + beta * d[q];
    __syncwarp();
    rr = rr_new;
  }
  return it;
}

// z = P^{-1} v: CG on each velocity block, lumped mass on the pressure.  On a
// single block and a small level (at most 2048 padded entries) the three CG
// solves run concurrently, warp w solving block w with warp-level
// synchronisation only; otherwise the team runs them in lockstep (cg3).
// cgf holds 9 scratch fields (3 per block).
__device__ inline int precond(const Ctx& C, const V4& v, const V4& z, double* const* cgf, int cg_max,
                              double cg_rtol) {
  __shared__ int its_sh[3];
  int its = 0;
  const int warp = threadIdx.x >> 5;
  const bool par = C.T.nblocks == 1 && blockDim.x >= 96 && C.L.nalloc <= 2048;
  if (par) {
    if (warp < 3) {
      const int n = cg_warp(C, v.c[warp], z.c[warp], cgf[3 * warp], cgf[3 * warp + 1], cgf[3 * warp + 2], cg_max,
                            cg_rtol);
      if ((threadIdx.x & 31) == 0) its_sh[warp] = n;
    }
  } else {
    V4 vu = v, zu = z;
    its = cg3(C, vu, zu, cgf, cg_max, cg_rtol);
  }
  const LevelDev<double>& L = C.L;
  for (int64_t q = C.T.rank(); q < C.n; q += C.T.size()) {
    int i, j, k;
    decode(L, q, i, j, k);
    const int64_t c = pidx(L.px, L.pxy, i, j, k);
    const uint8_t fl = L.flags[c];
    z.c[3][c] = (fl & F_ACT) ? v.c[3][c] / lumped_mass(L, c, fl) : 0.0;
  }
  C.T.sync();
  if (par) its = its_sh[0] + its_sh[1] + its_sh[2];
  C.T.sync();
  return its;
}

// (U, P) += PMINRES correction of the residual equation on level L; every
// thread of the team must call it.  scratch: COARSE_FIELDS fields of L.
__device__ inline void minres_team(const Team& T, const LevelDev<double>& L, double* scratch, const CoarseParams& prm,
                                   double* info) {
  Ctx C{L, T, (int64_t)L.nx * L.ny * L.nz};
  const int64_t na = L.nalloc;
  auto vec = [&](int first) {
    V4 v;
    for (int f = 0; f < 4; ++f) v.c[f] = scratch + (int64_t)(first + f) * na;
    return v;
  };
  // 11 vectors of 4 fields + 1 CG field = 45 fields (of COARSE_FIELDS)
  V4 b = vec(0), x = vec(4), Kz = vec(8);
  V4 vv[3] = {vec(12), vec(16), vec(20)};  // v_prev, v, v_next (rotating)
  V4 zz[2] = {vec(24), vec(28)};            // z, z_next
  V4 ww[3] = {vec(32), vec(36), vec(40)};  // w_prev, w, w_next
  double* cr = scratch + 44 * na;
  // CG scratch: b and Kz are dead whenever the preconditioner runs
  double* cgf[9] = {Kz.c[0], Kz.c[1], Kz.c[2], Kz.c[3], b.c[0], b.c[1], b.c[2], b.c[3], cr};
  for (int64_t q = T.rank(); q < 44 * na; q += T.size()) scratch[q] = 0.0;
  T.sync();

  // b = (F, G) - K (U, P): the residual equation of the current iterate
  V4 up;
  up.c[0] = L.u[0];
  up.c[1] = L.u[1];
  up.c[2] = L.u[2];
  up.c[3] = L.p;
  applyK(C, up, Kz);
  for (int64_t q = T.rank(); q < na; q += T.size()) {
    const uint8_t fl = L.flags[q];
    for (int d = 0; d < 3; ++d) b.c[d][q] = (fl & F_VFREE) ? L.f[d][q] - Kz.c[d][q] : 0.0;
    b.c[3][q] = (fl & F_ACT) ? L.g[q] - Kz.c[3][q] : 0.0;
  }
  T.sync();

  int iv_prev = 0, iv = 1, iv_next = 2, iz = 0, iz_next = 1, iw_prev = 0, iw = 1, iw_next = 2;
  // v_1 = b, z_1 = P^{-1} v_1
  for (int f = 0; f < 4; ++f)
    for (int64_t q = T.rank(); q < na; q += T.size()) vv[iv].c[f][q] = b.c[f][q];
  T.sync();
  int cg_total = precond(C, vv[iv], zz[iz], cgf, prm.cg_max, prm.cg_rtol);
  double gamma = sqrt(fmax(dot4(C, zz[iz], vv[iv]), 0.0));
  int its = 0;
  double rel = 0.0;
  if (gamma > 0.0) {
    const double gamma1 = gamma;
    double gamma_prev = 1.0, eta = gamma;
    double c_prev = 1.0, cc = 1.0, s_prev = 0.0, ss = 0.0;
    for (; its < prm.minres_max;) {
      for (int f = 0; f < 4; ++f)
        for (int64_t q = T.rank(); q < na; q += T.size()) zz[iz].c[f][q] /= gamma;
      T.sync();
      applyK(C, zz[iz], Kz);
      const double delta = dot4(C, Kz, zz[iz]);
      const double r1 = delta / gamma, r2 = gamma / gamma_prev;
      for (int f = 0; f < 4; ++f)
        for (int64_t q = T.rank(); q < na; q += T.size())
          vv[iv_next].c[f][q] = Kz.c[f][q] - r1 * vv[iv].c[f][q] - r2 * vv[iv_prev].c[f][q];
      T.sync();
      cg_total += precond(C, vv[iv_next], zz[iz_next], cgf, prm.cg_max, prm.cg_rtol);
      const double gamma_next = sqrt(fmax(dot4(C, zz[iz_next], vv[iv_next]), 0.0));
      const double a0 = cc * delta - c_prev * ss * gamma;
      const double a1 = sqrt(a0 * a0 + gamma_next * gamma_next);
      const double a2 = ss * delta + c_prev * cc * gamma;
      const double a3 = s_prev * gamma;
      if (a1 == 0.0) break;
      const double c_next = a0 / a1, s_next = gamma_next / a1;
      const double step = c_next * eta;
      for (int f = 0; f < 4; ++f)
        for (int64_t q = T.rank(); q < na; q += T.size()) {
          const double wn = (zz[iz].c[f][q] - a3 * ww[iw_prev].c[f][q] - a2 * ww[iw].c[f][q]) / a1;
          ww[iw_next].c[f][q] = wn;
          x.c[f][q] += step * wn;
        }
      T.sync();
      eta = -s_next * eta;
      ++its;
      // shift the recurrences
      int t = iv_prev;
      iv_prev = iv;
      iv = iv_next;
      iv_next = t;
      t = iz;
      iz = iz_next;
      iz_next = t;
      t = iw_prev;
      iw_prev = iw;
      iw = iw_next;
      iw_next = t;
      gamma_prev = gamma;
      gamma = gamma_next;
      c_prev = cc;
      cc = c_next;
      s_prev = ss;
      ss = s_next;
      rel = fabs(eta) / gamma1;
      if (fabs(eta) <= prm.minres_rtol * gamma1 || gamma == 0.0) break;
    }
  }
  // (U, P) += x
  for (int64_t q = T.rank(); q < na; q += T.size()) {
    L.u[0][q] += x.c[0][q];
    L.u[1][q] += x.c[1][q];
    L.u[2][q] += x.c[2][q];
    L.p[q] += x.c[3][q];
  }
  if (T.rank() == 0 && info) {
    info[0] = (double)its;
    info[1] = rel;
    info[2] = (double)cg_total;
  }}

}  // namespace coarse
}  // namespace hhg
