// Coarse-grid solver of the all-at-once multigrid (Sec. 3.7) as a routine of
// one team (a thread-block cluster, or one block; hhg_team.cuh): MINRES on the
// full saddle-point system, preconditioned block-diagonally (Sec. 3.2) with a
// CG solve on each velocity block of A and the inverse lumped pressure mass.
// Always FP64, on the compact unknown vector x = (u_0, u_1, u_2, p) of the
// coarsest level with K and A in CSR (CoarseSys), so no work is spent on the
// ghost frame, Dirichlet nodes or inactive nodes of the lattice.  Loops have
// fixed upper trip counts (max iterations).  Used by the coarse-solve kernel
// and by the fused coarse-levels cycle.
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

struct Ctx {
  CoarseSys S;
  Team T;
  int n;  // 3 nv + np
};

__device__ __forceinline__ double csr_row(const int32_t* ptr, const int32_t* col, const double* val, int r,
                                          const double* x) {
  double s = 0.0;
  const int e = ptr[r + 1];
  for (int k = ptr[r]; k < e; ++k) s += val[k] * x[col[k]];
  return s;
}

__device__ inline double dot(const Ctx& C, const double* a, const double* b) {
  double s = 0;
  for (int q = (int)C.T.rank(); q < C.n; q += (int)C.T.size()) s += a[q] * b[q];
  return team_sum1(C.T, s);
}

// y = K x
__device__ inline void applyK(const Ctx& C, const double* x, double* y) {
  for (int r = (int)C.T.rank(); r < C.n; r += (int)C.T.size()) y[r] = csr_row(C.S.kptr, C.S.kcol, C.S.kval, r, x);
  C.T.sync();
}

// x_d = CG(A, b_d) from zero for the three velocity blocks in lockstep over
// the team: each block follows the stopping rule of the single CG on its own
// (it stops before an iteration when r.r <= rtol^2 r0.r0 or r.r = 0, or when
// d.Ad = 0), the others go on; sums of the three blocks share one team
// reduction.  b, x: 3 nv entries; cg: 9 nv scratch (r, d, A d per block).
// Returns the iterations summed over the blocks.
__device__ inline int cg3(const Ctx& C, const double* b, double* x, double* cg, int max_it, double rtol) {
  const int nv = C.S.nv;
  double* R = cg;
  double* D = cg + 3 * nv;
  double* Q = cg + 6 * nv;
  for (int q = (int)C.T.rank(); q < 3 * nv; q += (int)C.T.size()) {
    x[q] = 0.0;
    R[q] = b[q];
    D[q] = b[q];
    Q[q] = 0.0;
  }
  C.T.sync();
  double rr[3] = {0, 0, 0};
  for (int q = (int)C.T.rank(); q < nv; q += (int)C.T.size())
#pragma unroll
    for (int d = 0; d < 3; ++d) rr[d] += R[d * nv + q] * R[d * nv + q];
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
    for (int q = (int)C.T.rank(); q < nv; q += (int)C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) Q[d * nv + q] = csr_row(C.S.aptr, C.S.acol, C.S.aval, q, D + d * nv);
    C.T.sync();
    double dq[3] = {0, 0, 0};
    for (int q = (int)C.T.rank(); q < nv; q += (int)C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) dq[d] += D[d * nv + q] * Q[d * nv + q];
    team_sum<3>(C.T, dq);
    double alpha[3];
    for (int d = 0; d < 3; ++d) {
      if (run[d] && dq[d] == 0.0) run[d] = false;
      alpha[d] = run[d] ? rr[d] / dq[d] : 0.0;
    }
    double rn[3] = {0, 0, 0};
    for (int q = (int)C.T.rank(); q < nv; q += (int)C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) {
          const int i = d * nv + q;
          x[i] += alpha[d] * D[i];
          R[i] -= alpha[d] * Q[i];
          rn[d] += R[i] * R[i];
        }
    team_sum<3>(C.T, rn);
    double beta[3];
    for (int d = 0; d < 3; ++d) beta[d] = run[d] ? rn[d] / rr[d] : 0.0;
    for (int q = (int)C.T.rank(); q < nv; q += (int)C.T.size())
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (run[d]) D[d * nv + q] = R[d * nv + q] + beta[d] * D[d * nv + q];
    C.T.sync();
    for (int d = 0; d < 3; ++d)
      if (run[d]) {
        rr[d] = rn[d];
        ++its;
      }
  }
  return its;
}

// x = CG(A, b) from zero on the coupled D-form velocity block (3 nv rows of
// A in CSR) over the team, same stopping rule; cg: 9 nv scratch.
__device__ inline int cg_coupled(const Ctx& C, const double* b, double* x, double* cg, int max_it, double rtol) {
  const int n = 3 * C.S.nv;
  double* R = cg;
  double* D = cg + n;
  double* Q = cg + 2 * n;
  double rr = 0.0;
  for (int q = (int)C.T.rank(); q < n; q += (int)C.T.size()) {
    x[q] = 0.0;
    R[q] = b[q];
    D[q] = b[q];
    rr += b[q] * b[q];
  }
  rr = team_sum1(C.T, rr);
  const double stop = rtol * rtol * rr;
  int it = 0;
  for (; it < max_it; ++it) {
    if (rr <= stop || rr == 0.0) break;
    double dq = 0.0;
    for (int q = (int)C.T.rank(); q < n; q += (int)C.T.size()) {
      const double aq = csr_row(C.S.aptr, C.S.acol, C.S.aval, q, D);
      Q[q] = aq;
      dq += D[q] * aq;
    }
    dq = team_sum1(C.T, dq);
    if (dq == 0.0) break;
    const double alpha = rr / dq;
    double rn = 0.0;
    for (int q = (int)C.T.rank(); q < n; q += (int)C.T.size()) {
      x[q] += alpha * D[q];
      R[q] -= alpha * Q[q];
      rn += R[q] * R[q];
    }
    rn = team_sum1(C.T, rn);
    const double beta = rn / rr;
    for (int q = (int)C.T.rank(); q < n; q += (int)C.T.size()) D[q] = R[q] + beta * D[q];
    C.T.sync();
    rr = rn;
  }
  return it;
}

// ---- warp-level CG: the three velocity blocks are solved concurrently ------

// Sum over the warp, the same value in every lane (shuffle tree, lane 0 broadcast).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// x = CG(A, b) from zero by one warp (same stopping rule as cg3).
__device__ inline int cg_warp(const CoarseSys& S, const double* b, double* x, double* r, double* d, double* w,
                              int max_it, double rtol) {
  const int lane = threadIdx.x & 31, nv = S.nv;
  double rr = 0.0;
  for (int q = lane; q < nv; q += 32) {
    x[q] = 0.0;
    r[q] = b[q];
    d[q] = b[q];
    rr += b[q] * b[q];
  }
  rr = warp_sum(rr);
  __syncwarp();
  const double stop = rtol * rtol * rr;
  int it = 0;
  for (; it < max_it; ++it) {
    if (rr <= stop || rr == 0.0) break;
    double dq = 0.0;
    for (int q = lane; q < nv; q += 32) {
      const double aq = csr_row(S.aptr, S.acol, S.aval, q, d);
      w[q] = aq;
      dq += d[q] * aq;
    }
    dq = warp_sum(dq);
    if (dq == 0.0) break;
    const double alpha = rr / dq;
    double rn = 0.0;
    for (int q = lane; q < nv; q += 32) {
      x[q] += alpha * d[q];
      const double rq = r[q] - alpha * w[q];
      r[q] = rq;
      rn += rq * rq;
    }
    rn = warp_sum(rn);
    const double beta = rn / rr;
    // every lane has read d (the products above) before any lane rewrites it
    __syncwarp();
    for (int q = lane; q < nv; q += 32) d[q] = r[q] + beta * d[q];
    __syncwarp();
    rr = rn;
  }
  return it;
}

// Largest velocity block solved by one warp in the single-block solver.
constexpr int WARP_CG_MAX_NV = 1024;

// z = P^{-1} v: CG on each velocity block, lumped mass on the pressure.  On a
// single block with small blocks the three CG solves run concurrently, warp
// w solving block w with warp-level synchronisation only; otherwise the team
// runs them in lockstep (cg3).  cg holds 9 nv scratch entries.
__device__ inline int precond(const Ctx& C, const double* v, double* z, double* cg, int cg_max, double cg_rtol) {
  __shared__ int its_sh[3];
  int its = 0;
  const int nv = C.S.nv;
  const int warp = threadIdx.x >> 5;
  const bool par = !C.S.coupled && C.T.nblocks == 1 && blockDim.x >= 96 && nv <= WARP_CG_MAX_NV;
  if (C.S.coupled) {
    its = cg_coupled(C, v, z, cg, cg_max, cg_rtol);
  } else if (par) {
    if (warp < 3) {
      const int n = cg_warp(C.S, v + warp * nv, z + warp * nv, cg + 3 * warp * nv, cg + (3 * warp + 1) * nv,
                            cg + (3 * warp + 2) * nv, cg_max, cg_rtol);
      if ((threadIdx.x & 31) == 0) its_sh[warp] = n;
    }
  } else {
    its = cg3(C, v, z, cg, cg_max, cg_rtol);
  }
  for (int q = (int)C.T.rank(); q < C.S.np; q += (int)C.T.size()) z[3 * nv + q] = v[3 * nv + q] / C.S.mass[q];
  C.T.sync();
  if (par) its = its_sh[0] + its_sh[1] + its_sh[2];
  C.T.sync();
  return its;
}

// (U, P) += PMINRES correction of the residual equation (F, G) - K (U, P) on
// the coarsest level L (fields of type T, the solve in FP64); every thread of
// the team must call it.  scratch: coarse_scratch_doubles(S) entries.
template <class T>
__device__ inline void minres_team(const Team& tm, const CoarseSys& S, const LevelDev<T>& L, double* scratch,
                                   const CoarseParams& prm, double* info) {
  const int nv = S.nv, n = 3 * S.nv + S.np;
  Ctx C{S, tm, n};
  double* vec[11];
  for (int f = 0; f < 11; ++f) vec[f] = scratch + (int64_t)f * n;
  double* cg = scratch + (int64_t)11 * n;
  double *b = vec[0], *x = vec[1], *Kz = vec[2];
  double* vv[3] = {vec[3], vec[4], vec[5]};  // v_prev, v, v_next (rotating)
  double* zz[2] = {vec[6], vec[7]};          // z, z_next
  double* ww[3] = {vec[8], vec[9], vec[10]};  // w_prev, w, w_next

  // gather (U, P) into Kz and (F, G) into b; zero x, v_prev, w_prev, w
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    double up, fg;
    if (q < 3 * nv) {
      const int d = q / nv;
      const int c = S.vidx[q - d * nv];
      up = (double)L.u[d][c];
      if (L.flags[c] & F_SLIP) {
        // the admissible part of f at a free-slip node: the assembled rows
        // carry the identity in the constrained directions (Sec. 6.1)
        T fv[3] = {L.f[0][c], L.f[1][c], L.f[2][c]};
        slip_project(class_row(L, c), fv);
        fg = (double)fv[d];
      } else {
        fg = (double)L.f[d][c];
      }
    } else {
      const int c = S.pidx[q - 3 * nv];
      up = (double)L.p[c];
      fg = (double)L.g[c];
    }
    Kz[q] = up;
    b[q] = fg;
    x[q] = 0.0;
    vv[0][q] = 0.0;
    ww[0][q] = 0.0;
    ww[1][q] = 0.0;
  }
  tm.sync();
  // b = (F, G) - K (U, P), v_1 = b
  for (int r = (int)tm.rank(); r < n; r += (int)tm.size()) {
    const double br = b[r] - csr_row(S.kptr, S.kcol, S.kval, r, Kz);
    b[r] = br;
    vv[1][r] = br;
  }
  tm.sync();

  int iv_prev = 0, iv = 1, iv_next = 2, iz = 0, iz_next = 1, iw_prev = 0, iw = 1, iw_next = 2;
  int cg_total = precond(C, vv[iv], zz[iz], cg, prm.cg_max, prm.cg_rtol);
  double gamma = sqrt(fmax(dot(C, zz[iz], vv[iv]), 0.0));
  int its = 0;
  double rel = 0.0;
  if (gamma > 0.0) {
    const double gamma1 = gamma;
    double gamma_prev = 1.0, eta = gamma;
    double c_prev = 1.0, cc = 1.0, s_prev = 0.0, ss = 0.0;
    for (; its < prm.minres_max;) {
      for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) zz[iz][q] /= gamma;
      tm.sync();
      applyK(C, zz[iz], Kz);
      const double delta = dot(C, Kz, zz[iz]);
      const double r1 = delta / gamma, r2 = gamma / gamma_prev;
      for (int q = (int)tm.rank(); q < n; q += (int)tm.size())
        vv[iv_next][q] = Kz[q] - r1 * vv[iv][q] - r2 * vv[iv_prev][q];
      tm.sync();
      cg_total += precond(C, vv[iv_next], zz[iz_next], cg, prm.cg_max, prm.cg_rtol);
      const double gamma_next = sqrt(fmax(dot(C, zz[iz_next], vv[iv_next]), 0.0));
      const double a0 = cc * delta - c_prev * ss * gamma;
      const double a1 = sqrt(a0 * a0 + gamma_next * gamma_next);
      const double a2 = ss * delta + c_prev * cc * gamma;
      const double a3 = s_prev * gamma;
      if (a1 == 0.0) break;
      const double c_next = a0 / a1, s_next = gamma_next / a1;
      const double step = c_next * eta;
      for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
        const double wn = (zz[iz][q] - a3 * ww[iw_prev][q] - a2 * ww[iw][q]) / a1;
        ww[iw_next][q] = wn;
        x[q] += step * wn;
      }
      tm.sync();
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
  for (int q = (int)tm.rank(); q < n; q += (int)tm.size()) {
    if (q < 3 * nv) {
      const int d = q / nv;
      const int c = S.vidx[q - d * nv];
      L.u[d][c] = (T)((double)L.u[d][c] + x[q]);
    } else {
      const int c = S.pidx[q - 3 * nv];
      L.p[c] = (T)((double)L.p[c] + x[q]);
    }
  }
  if (tm.rank() == 0 && info) {
    info[0] = (double)its;
    info[1] = rel;
    info[2] = (double)cg_total;
  }
}

}  // namespace coarse
}  // namespace hhg
