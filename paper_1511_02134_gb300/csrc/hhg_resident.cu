// Cluster-resident cycle of the coarse levels (Sec. 3.5 V_var cycle below a
// mid-sized level, Sec. 3.7 coarse solve).
//
// On the small levels of the hierarchy a colour phase updates a few thousand
// nodes, and its cost is the latency of one launch or of the dependent loads
// from L2.  Here the levels lv[1..nres] are held in the shared memory of one
// thread-block cluster for the whole sub-cycle: every level is split into
// runs of z-planes, one run per CTA, each CTA updates the nodes of its own
// planes, and reads neighbours on other CTAs' planes through distributed
// shared memory.  Phases are separated by the cluster barrier (release /
// acquire at cluster scope).  The coarsest level stays in global memory, where
// the first CTA runs the coarse solve (hhg_coarse_block.cuh) while the others
// wait at the barrier.
//
// The per-node arithmetic is the view form of the grid kernels' bodies
// (hhg_node_ops.cuh): the node's own fields are reached through a LevelDev
// whose field pointers point at the node's plane, its neighbours through
// plane-pointer tables, the boundary-class rows from a copy of the level's
// table in shared memory.
#include <cooperative_groups.h>

#include <algorithm>

#include "hhg_coarse_block.cuh"
#include "hhg_kernels.h"
#include "hhg_node_ops.cuh"
#include "hhg_team.cuh"

namespace hhg {

namespace {

namespace cg = cooperative_groups;

constexpr int RT = 512;  // threads per CTA

__host__ __device__ inline uint32_t align16(uint64_t x) { return (uint32_t)((x + 15) & ~(uint64_t)15); }

// Neighbour view over a plane-pointer table row: row[z] is the generic
// address (local or another CTA's shared memory) of padded plane z.
template <class T>
struct DNb {
  T* const* row;
  int z, xy, dxm, dxp, px;
  __device__ __forceinline__ T operator()(int dx, int dy, int dz) const {
    return row[z + dz][xy + (dx < 0 ? dxm : (dx > 0 ? dxp : 0)) + px * dy];
  }
};

// In-plane position of node (i, j) of a level and the steps to its
// x-neighbours (rows grouped by x mod 4, hhg_common.h).
struct InPlane {
  int xy, dxm, dxp;
};

template <class T>
__device__ __forceinline__ InPlane in_plane(const LevelDev<T>& L, int i, int j) {
  return InPlane{(int)(L.px * (j + 1) + row_pos(i + 1, L.px)), (int)row_step_minus(i + 1, L.px),
                 (int)row_step_plus(i + 1, L.px)};
}

template <class T>
struct Res {
  const ResidentCycle<T>& S;
  unsigned char* sm;
  unsigned rank;

  __device__ __forceinline__ void* const* table(int q) const {
    return reinterpret_cast<void* const*>(sm + S.tab[q]);
  }
  template <class E>
  __device__ __forceinline__ E* row_ptr(int q, int f, int z) const {
    return reinterpret_cast<E*>(table(q)[f * (S.lv[q].nz + 2) + z]);
  }
  // The level with its field pointers at padded plane z (node plane z - 1):
  // node (i, j) of that plane is entry in_plane(L, i, j).xy.
  __device__ __forceinline__ LevelDev<T> at_plane(int q, int z) const {
    LevelDev<T> L = S.lv[q];
    L.wt = reinterpret_cast<const T*>(sm + S.wts[q]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      L.u[d] = row_ptr<T>(q, d, z);
      L.f[d] = row_ptr<T>(q, 4 + d, z);
    }
    L.p = row_ptr<T>(q, 3, z);
    L.g = row_ptr<T>(q, 7, z);
#pragma unroll
    for (int d = 0; d < 3; ++d) L.r[d] = row_ptr<T>(q, 8 + d, z);
    L.rp = row_ptr<T>(q, 11, z);
    L.flags = row_ptr<const uint8_t>(q, RES_FIELDS, z);
    L.cls = row_ptr<const uint16_t>(q, RES_FIELDS + 1, z);
    return L;
  }
  // Offsets of this CTA's part of list l of level q in its copy (loc(q)[l])
  // and in the level's list array (loc(q)[RES_LISTS + 1 + l]).
  __device__ __forceinline__ int* loc(int q) const {
    return reinterpret_cast<int*>(sm + S.lofs) + q * 2 * (RES_LISTS + 1);
  }
  __device__ __forceinline__ DNb<T> view(int q, int f, int z, const InPlane& at) const {
    void* const* t = table(q) + f * (S.lv[q].nz + 2);
    return DNb<T>{reinterpret_cast<T* const*>(t), z, at.xy, at.dxm, at.dxp, (int)S.lv[q].px};
  }
};

__device__ __forceinline__ void cluster_sync() { cg::this_cluster().sync(); }

// End of a phase of level q: the cluster barrier when the level is spread
// over several CTAs, the block barrier when the first CTA holds it alone
// (the other CTAs skip the level's phases).
template <class T>
__device__ __forceinline__ void level_sync(const ResidentCycle<T>& S, int q) {
  if (S.nbq[q] > 1)
    cluster_sync();
  else
    __syncthreads();
}

// ---- set-up: plane tables, zero plane, flags / classes, top-level fields ------

// First position in list[a, b) (entries (k << 20) | (j << 10) | i, sorted by
// k) whose plane k is at least kk.
__device__ __forceinline__ int first_on_plane(const int32_t* list, int a, int b, int kk) {
  while (a < b) {
    const int m = (a + b) >> 1;
    if ((list[m] >> 20) < kk)
      a = m + 1;
    else
      b = m;
  }
  return a;
}

template <class T>
__device__ void r_setup(const Res<T>& R) {
  const ResidentCycle<T>& S = R.S;
  cg::cluster_group cl = cg::this_cluster();
  // zero everything this CTA holds (blocks and zero plane)
  {
    uint4* z = reinterpret_cast<uint4*>(R.sm + S.zero);
    const uint4* e = reinterpret_cast<const uint4*>(R.sm + S.smem);
    for (uint4* p = z + threadIdx.x; p < e; p += blockDim.x) *p = make_uint4(0, 0, 0, 0);
  }
  for (int q = 1; q <= S.nres; ++q) {
    const LevelDev<T>& L = S.lv[q];
    const int pz = L.nz + 2;
    const int64_t plane = L.pxy;
    const int64_t fb = (int64_t)S.maxpl[q] * plane;  // entries per field block
    void** tab = reinterpret_cast<void**>(R.sm + S.tab[q]);
    for (int e = threadIdx.x; e < RES_TAB_FIELDS * pz; e += blockDim.x) {
      const int f = e / pz, z = e - f * pz;
      void* ptr = R.sm + S.zero;
      if (z >= 1 && z <= L.nz) {
        const int k = z - 1;
        const unsigned r = (unsigned)(((int64_t)k * S.nbq[q]) / L.nz);
        const int64_t lp = k - S.kb[q][r];
        unsigned char* base = R.sm + S.blk[q];
        unsigned char* loc;
        if (f < RES_FIELDS)
          loc = base + sizeof(T) * (f * fb + lp * plane);
        else if (f == RES_FIELDS)
          loc = base + sizeof(T) * RES_FIELDS * fb + lp * plane;
        else
          loc = base + align16(sizeof(T) * RES_FIELDS * fb + fb) + 2 * lp * plane;
        // own planes through the CTA's own shared window, others' through the cluster's
        ptr = r == R.rank ? (void*)loc : cl.map_shared_rank(loc, r);
      }
      tab[e] = ptr;
    }
  }
  // this CTA's part of the node lists: the entries of planes [k0, k1) of
  // every list (each sorted by plane), found by bisection on the plane
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    for (int q = 1; q <= S.nres; ++q) {
      if (!S.lists[q]) continue;
      int lo = 0, len = 0;
      if (l < RES_LISTS) {
        lo = first_on_plane(S.lists[q], S.loff[q][l], S.loff[q][l + 1], S.kb[q][R.rank]);
        len = first_on_plane(S.lists[q], lo, S.loff[q][l + 1], S.kb[q][R.rank + 1]) - lo;
      }
      int x = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
      }
      int* lc = R.loc(q);
      if (l < RES_LISTS) {
        lc[l] = x - len;
        lc[RES_LISTS + 1 + l] = lo;
      }
      if (l == RES_LISTS - 1) lc[RES_LISTS] = x;
    }
  }
  __syncthreads();
  for (int q = 1; q <= S.nres; ++q) {
    if (!S.lists[q]) continue;
    const int* lc = R.loc(q);
    int32_t* dst = reinterpret_cast<int32_t*>(R.sm + S.lst[q]);
    for (int l = 0; l < RES_LISTS; ++l) {
      const int n = lc[l + 1] - lc[l];
      const int32_t* src = S.lists[q] + lc[RES_LISTS + 1 + l];
      for (int e = threadIdx.x; e < n; e += blockDim.x) dst[lc[l] + e] = src[e];
    }
  }
  // class-row tables of the resident levels
  for (int q = 1; q <= S.nres; ++q) {
    T* w = reinterpret_cast<T*>(R.sm + S.wts[q]);
    const int n = (S.ncls[q] + 1) * W_STRIDE;
    for (int e = threadIdx.x; e < n; e += blockDim.x) w[e] = S.lv[q].wt[e];
  }
  __syncthreads();
  // flags and classes of every resident level, fields of the top level
  for (int q = 1; q <= S.nres; ++q) {
    const LevelDev<T>& L = S.lv[q];
    const int k0 = S.kb[q][R.rank], k1 = S.kb[q][R.rank + 1];
    const int64_t plane = L.pxy, fb = (int64_t)S.maxpl[q] * plane;
    const int64_t n = (int64_t)(k1 - k0) * plane;
    const int64_t g0 = (int64_t)(k0 + 1) * plane;  // first padded entry of plane k0
    unsigned char* base = R.sm + S.blk[q];
    uint8_t* fl = base + sizeof(T) * RES_FIELDS * fb;
    uint16_t* cs = reinterpret_cast<uint16_t*>(base + align16(sizeof(T) * RES_FIELDS * fb + fb));
    T* fld = reinterpret_cast<T*>(base);
    const bool top = q == S.nres;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      fl[e] = L.flags[g0 + e];
      cs[e] = L.cls[g0 + e];
      if (top) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          fld[d * fb + e] = L.u[d][g0 + e];
          fld[(4 + d) * fb + e] = L.f[d][g0 + e];
        }
        fld[3 * fb + e] = L.p[g0 + e];
        fld[7 * fb + e] = L.g[g0 + e];
      }
    }
  }
  cluster_sync();
}

// u, p of the top level back to global memory
template <class T>
__device__ void r_writeback(const Res<T>& R) {
  const ResidentCycle<T>& S = R.S;
  const int q = S.nres;
  const LevelDev<T>& L = S.lv[q];
  const int k0 = S.kb[q][R.rank], k1 = S.kb[q][R.rank + 1];
  const int64_t plane = L.pxy, fb = (int64_t)S.maxpl[q] * plane;
  const int64_t n = (int64_t)(k1 - k0) * plane;
  const int64_t g0 = (int64_t)(k0 + 1) * plane;
  const T* fld = reinterpret_cast<const T*>(R.sm + S.blk[q]);
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) L.u[d][g0 + e] = fld[d * fb + e];
    L.p[g0 + e] = fld[3 * fb + e];
  }
}

// ---- phases --------------------------------------------------------------------

// One colour phase of level q on this CTA's planes: velocity Gauss-Seidel with
// f - B^T p formed at the node (what = 0), the relaxed pressure update with
// B u - g (what = 1), or both at each node (what = 2: the last velocity
// colour of a step with the first pressure colour).
template <class T>
__device__ void r_colour(const Res<T>& R, int q, int colour, int what) {
  const ResidentCycle<T>& S = R.S;
  const LevelDev<T>& L = S.lv[q];
  const int k0 = S.kb[q][R.rank], k1 = S.kb[q][R.rank + 1];
  const int nq = (L.nx + 3) / 4;
  const int n = (k1 - k0) * L.ny * nq;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int tq = t % nq;
    const int j = (t / nq) % L.ny;
    const int k = k0 + t / (nq * L.ny);
    const int i = ((colour - j - k) & 3) + 4 * tq;
    if (i >= L.nx) continue;
    const LevelDev<T> Ln = R.at_plane(q, k + 1);
    const InPlane at = in_plane(L, i, j);
    const int c = at.xy;
    const DNb<T> u[3] = {R.view(q, 0, k + 1, at), R.view(q, 1, k + 1, at), R.view(q, 2, k + 1, at)};
    const DNb<T> p = R.view(q, 3, k + 1, at);
    if (what != 1) node_vel_gs_rhs_v<true>(Ln, c, u, p, S.inv6nuh[q]);
    if (what != 0) node_pres_gs_rhs_v<true>(Ln, c, u, p, S.omc[q]);
  }
  level_sync(S, q);
}

// The same phase over this CTA's node lists (what = KIND: 0 velocity, 1
// pressure, 2 both): the regular nodes of the colour, then its boundary
// nodes, so that a warp takes one update form and no node is skipped.  KIND
// 2 walks the pressure lists (every velocity node carries a pressure, and
// every regular node a velocity).
template <int KIND, class T>
__device__ void r_colour_list(const Res<T>& R, int q, int colour) {
  const ResidentCycle<T>& S = R.S;
  const LevelDev<T>& L = S.lv[q];
  const int* lc = R.loc(q);
  const uint32_t* ls = reinterpret_cast<const uint32_t*>(R.sm + S.lst[q]);
  const int l = 8 * (KIND != 0) + 2 * colour;
  const int a1 = lc[l + 1], a2 = lc[l + 2];
  for (int t = lc[l] + threadIdx.x; t < a2; t += blockDim.x) {
    const uint32_t e = ls[t];
    const int i = e & 1023, j = (e >> 10) & 1023, k = e >> 20;
    const LevelDev<T> Ln = R.at_plane(q, k + 1);
    const InPlane at = in_plane(L, i, j);
    const int c = at.xy;
    const DNb<T> u[3] = {R.view(q, 0, k + 1, at), R.view(q, 1, k + 1, at), R.view(q, 2, k + 1, at)};
    const DNb<T> p = R.view(q, 3, k + 1, at);
    if (KIND != 1) {
      if (t < a1) {
        T reg[3];
        vel_rhs_regular(Ln, c, u, p, S.inv6nuh[q], reg);
#pragma unroll
        for (int d = 0; d < 3; ++d) Ln.u[d][c] = reg[d];
      } else if (KIND == 0 || (Ln.flags[c] & F_VFREE)) {
        vel_rhs_irr(Ln, c, u, p);
      }
    }
    if (KIND != 0) {
      const T pc = p(0, 0, 0);
      if (t < a1)
        Ln.p[c] = pres_rhs_regular(Ln, c, u, p, pc, S.omc[q]);
      else
        pres_rhs_irr(Ln, c, u, p, pc);
    }
  }
  level_sync(S, q);
}

template <class T>
__device__ void r_uzawa(const Res<T>& R, int q) {
  if (R.S.nbq[q] == 1 && R.rank != 0) return;
  if (R.S.lists[q]) {
    for (int c = 0; c < 4; ++c) r_colour_list<0>(R, q, c);
    for (int c = 2; c >= 1; --c) r_colour_list<0>(R, q, c);
    r_colour_list<2>(R, q, 0);
    for (int c = 1; c < 4; ++c) r_colour_list<1>(R, q, c);
    return;
  }
  for (int c = 0; c < 4; ++c) r_colour(R, q, c, 0);
  for (int c = 2; c >= 1; --c) r_colour(R, q, c, 0);
  r_colour(R, q, 0, 2);
  for (int c = 1; c < 4; ++c) r_colour(R, q, c, 1);
}

// (RU, RP) of level q on this CTA's planes (node_residual).
template <class T>
__device__ void r_residual(const Res<T>& R, int q) {
  const ResidentCycle<T>& S = R.S;
  const LevelDev<T>& L = S.lv[q];
  const int k0 = S.kb[q][R.rank], k1 = S.kb[q][R.rank + 1];
  const int n = (k1 - k0) * L.ny * L.nx;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % L.nx;
    const int j = (t / L.nx) % L.ny;
    const int k = k0 + t / (L.nx * L.ny);
    const LevelDev<T> Ln = R.at_plane(q, k + 1);
    const InPlane at = in_plane(L, i, j);
    const int c = at.xy;
    const uint8_t fl = Ln.flags[c];
    const DNb<T> u[3] = {R.view(q, 0, k + 1, at), R.view(q, 1, k + 1, at), R.view(q, 2, k + 1, at)};
    T r[4];
    node_residual_v(Ln, c, fl, u, R.view(q, 3, k + 1, at), r);
#pragma unroll
    for (int d = 0; d < 3; ++d) Ln.r[d][c] = r[d];
    Ln.rp[c] = r[3];
  }
}

// (F, G) of level q - 1 = P^T (RU, RP) of level q, (U, P) of level q - 1 = 0
// (node_restrict).  The coarse level is resident (its nodes on this CTA's
// planes) or the coarsest level in global memory (its nodes shared by the
// team).
template <class T>
__device__ void r_restrict(const Res<T>& R, int q) {
  const ResidentCycle<T>& S = R.S;
  cluster_sync();  // the fine level's last phase may have run on the first CTA alone
  r_residual(R, q);
  cluster_sync();
  const LevelDev<T>& Lf = S.lv[q];
  const LevelDev<T>& Lc = S.lv[q - 1];
  const bool resident = q - 1 >= 1;
  int k0, k1, t0, ts;
  if (resident) {
    k0 = S.kb[q - 1][R.rank];
    k1 = S.kb[q - 1][R.rank + 1];
    t0 = threadIdx.x;
    ts = blockDim.x;
  } else {
    k0 = 0;
    k1 = Lc.nz;
    t0 = R.rank * blockDim.x + threadIdx.x;
    ts = S.nblocks * blockDim.x;
  }
  const int n = (k1 - k0) * Lc.ny * Lc.nx;
  for (int t = t0; t < n; t += ts) {
    const int I = t % Lc.nx;
    const int J = (t / Lc.nx) % Lc.ny;
    const int K = k0 + t / (Lc.nx * Lc.ny);
    const InPlane at = in_plane(Lf, 2 * I, 2 * J);
    T s[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const DNb<T> x = R.view(q, 8 + w, 2 * K + 1, at);
      // the 14 Kuhn neighbours: +-(e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3)
      T acc = 0;
      acc += x(1, 0, 0) + x(-1, 0, 0);
      acc += x(0, 1, 0) + x(0, -1, 0);
      acc += x(0, 0, 1) + x(0, 0, -1);
      acc += x(1, 1, 0) + x(-1, -1, 0);
      acc += x(0, 1, 1) + x(0, -1, -1);
      acc += x(1, 0, 1) + x(-1, 0, -1);
      acc += x(1, 1, 1) + x(-1, -1, -1);
      s[w] = x(0, 0, 0) + (T)0.5 * acc;
    }
    LevelDev<T> C;
    int64_t cc;
    if (resident) {
      C = R.at_plane(q - 1, K + 1);
      cc = in_plane(Lc, I, J).xy;
    } else {
      C = Lc;
      cc = pidx(Lc.px, Lc.pxy, I, J, K);
    }
    const uint8_t fl = C.flags[cc];
    const bool vf = fl & F_VFREE, ac = fl & F_ACT;
    if (fl & F_SLIP) slip_project(class_row(C, cc), s);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      C.f[d][cc] = vf ? s[d] : (T)0;
      C.u[d][cc] = (T)0;
    }
    C.g[cc] = ac ? s[3] : (T)0;
    C.p[cc] = (T)0;
  }
  cluster_sync();
}

// Fine (U, P) of level q += P (U, P) of level q - 1 (node_prolong_add).
template <class T>
__device__ void r_prolong(const Res<T>& R, int q) {
  const ResidentCycle<T>& S = R.S;
  cluster_sync();  // the coarse level's last phase may have run on the first CTA alone
  const LevelDev<T>& Lf = S.lv[q];
  const LevelDev<T>& Lc = S.lv[q - 1];
  const bool resident = q - 1 >= 1;
  const int k0 = S.kb[q][R.rank], k1 = S.kb[q][R.rank + 1];
  const int n = (k1 - k0) * Lf.ny * Lf.nx;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % Lf.nx;
    const int j = (t / Lf.nx) % Lf.ny;
    const int k = k0 + t / (Lf.nx * Lf.ny);
    const LevelDev<T> F = R.at_plane(q, k + 1);
    const int cf = in_plane(Lf, i, j).xy;
    const uint8_t fl = F.flags[cf];
    if (!(fl & F_ACT)) continue;
    const int a = i & 1, b = j & 1, e = k & 1;
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const bool mid = (a | b | e) != 0;
    const T* cu0[4];
    const T* cu1[4];
    int64_t c0, c1;
    if (resident) {
      const LevelDev<T> A = R.at_plane(q - 1, K + 1), B = R.at_plane(q - 1, K + e + 1);
      cu0[0] = A.u[0];
      cu0[1] = A.u[1];
      cu0[2] = A.u[2];
      cu0[3] = A.p;
      cu1[0] = B.u[0];
      cu1[1] = B.u[1];
      cu1[2] = B.u[2];
      cu1[3] = B.p;
      c0 = in_plane(Lc, I, J).xy;
      c1 = in_plane(Lc, I + a, J + b).xy;
    } else {
      cu0[0] = cu1[0] = Lc.u[0];
      cu0[1] = cu1[1] = Lc.u[1];
      cu0[2] = cu1[2] = Lc.u[2];
      cu0[3] = cu1[3] = Lc.p;
      c0 = pidx(Lc.px, Lc.pxy, I, J, K);
      c1 = pidx(Lc.px, Lc.pxy, I + a, J + b, K + e);
    }
    if (fl & F_VFREE) {
      T v[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] = mid ? (T)0.5 * (cu0[d][c0] + cu1[d][c1]) : cu0[d][c0];
      if (fl & F_SLIP) slip_project(class_row(F, cf), v);
#pragma unroll
      for (int d = 0; d < 3; ++d) F.u[d][cf] += v[d];
    }
    const T v = mid ? (T)0.5 * (cu0[3][c0] + cu1[3][c1]) : cu0[3][c0];
    F.p[cf] += v;
  }
  cluster_sync();
}

template <class T>
__device__ void r_coarse(const Res<T>& R) {
  const ResidentCycle<T>& S = R.S;
  cluster_sync();
  if (coarse_fits_block(S.cs)) {
    if (R.rank == 0) {
      coarse::minres_team(Team{1}, S.cs, S.lv[0], S.scratch, S.prm, S.info);
    }
  } else {
    coarse::minres_team(Team{S.nblocks}, S.cs, S.lv[0], S.scratch, S.prm, S.info);
  }
  cluster_sync();
}

template <class T>
__global__ void __launch_bounds__(RT) k_resident(const __grid_constant__ ResidentCycle<T> S) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char sm[];
  const Res<T> R{S, sm, blockIdx.x};
  r_setup(R);
  for (int q = S.nres; q >= 1; --q) {
    for (int s = 0; s < S.nu_pre[q]; ++s) r_uzawa(R, q);
    r_restrict(R, q);
  }
  r_coarse(R);
  for (int q = 1; q <= S.nres; ++q) {
    r_prolong(R, q);
    for (int s = 0; s < S.nu_post[q]; ++s) r_uzawa(R, q);
  }
  if (S.nbq[S.nres] == 1) __syncthreads();
  r_writeback(R);
}

}  // namespace

// Lays out the shared memory for per-level CTA counts nbq (cluster size the
// largest of them); returns the bytes per CTA.
template <class T>
uint64_t layout_resident(ResidentCycle<T>& S) {
  unsigned nb = 1;
  for (int q = 1; q <= S.nres; ++q) nb = std::max(nb, (unsigned)S.nbq[q]);
  S.nblocks = nb;
  uint64_t off = 0;
  for (int q = 1; q <= S.nres; ++q) {
    S.tab[q] = (uint32_t)off;
    off = align16(off + sizeof(void*) * RES_TAB_FIELDS * (uint64_t)(S.lv[q].nz + 2));
  }
  for (int q = 1; q <= S.nres; ++q) {
    S.wts[q] = (uint32_t)off;
    off = align16(off + sizeof(T) * (uint64_t)(S.ncls[q] + 1) * W_STRIDE);
  }
  int64_t zero_bytes = 0;
  for (int q = 1; q <= S.nres; ++q) {
    const LevelDev<T>& L = S.lv[q];
    const int nbq = S.nbq[q];
    int mx = 0;
    for (unsigned r = 0; r <= nb; ++r)
      S.kb[q][r] = r <= (unsigned)nbq ? (int)(((int64_t)r * L.nz + nbq - 1) / nbq) : L.nz;
    for (unsigned r = 0; r < nb; ++r) mx = std::max(mx, S.kb[q][r + 1] - S.kb[q][r]);
    S.maxpl[q] = mx;
    zero_bytes = std::max<int64_t>(zero_bytes, (int64_t)L.pxy * (int64_t)std::max<size_t>(sizeof(T), 2));
  }
  // node lists: every lattice node is in at most one velocity and one pressure list
  S.lofs = (uint32_t)off;
  off = align16(off + sizeof(int) * 2 * (RES_LISTS + 1) * (uint64_t)(S.nres + 1));
  for (int q = 1; q <= S.nres; ++q) {
    S.lst[q] = (uint32_t)off;
    if (S.lists[q]) off = align16(off + sizeof(int32_t) * 2 * (uint64_t)S.maxpl[q] * S.lv[q].nx * S.lv[q].ny);
  }
  S.zero = (uint32_t)off;
  off = align16(off + zero_bytes);
  for (int q = 1; q <= S.nres; ++q) {
    const int64_t fb = (int64_t)S.maxpl[q] * S.lv[q].pxy;
    S.blk[q] = (uint32_t)off;
    off = align16(off + align16(sizeof(T) * RES_FIELDS * fb + fb) + 2 * fb);
  }
  S.smem = (uint32_t)off;
  return off;
}

// Every level is spread over all max_ctas CTAs of the cluster.  Measured on
// GB300 (cube, levels 3-4 resident), a phase costs 1.8 us spread over 8 or 16
// CTAs and 2.4 us with each level on the fewest CTAs whose shared memory
// holds it (level 3 on one CTA with block barriers, level 4 on two): the
// cost is the instruction latency of one node update, and more CTAs put
// fewer nodes on each thread.
template <class T>
bool plan_resident(ResidentCycle<T>& S, size_t smem_limit, unsigned max_ctas) {
  if (S.nres < 1 || S.nres > RES_MAX_LEVELS || max_ctas < 1 || max_ctas > RES_MAX_CTAS) return false;
  for (int q = 1; q <= S.nres; ++q) S.nbq[q] = (int)max_ctas;
  return layout_resident(S) <= smem_limit;
}

template <class T>
cudaError_t launch_resident_cycle(const ResidentCycle<T>& S, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S.nblocks, 1, 1);
  cfg.blockDim = dim3(RT, 1, 1);
  cfg.dynamicSmemBytes = S.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = S.nblocks;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_resident<T>, S);
}

template <class T>
unsigned prepare_resident(size_t& smem_limit) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k_resident<T>);
  smem_limit = optin > (int)fa.sharedSizeBytes ? (size_t)(optin - fa.sharedSizeBytes) : 0;
  cudaFuncSetAttribute(k_resident<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit);
  unsigned nb = 8;
  if (cudaFuncSetAttribute(k_resident<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(RT, 1, 1);
    cfg.dynamicSmemBytes = smem_limit;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_resident<T>, &cfg) == cudaSuccess && n >= 1) nb = 16;
  }
  cudaGetLastError();
  return nb;
}

template bool plan_resident<float>(ResidentCycle<float>&, size_t, unsigned);
template bool plan_resident<double>(ResidentCycle<double>&, size_t, unsigned);
template cudaError_t launch_resident_cycle<float>(const ResidentCycle<float>&, cudaStream_t);
template cudaError_t launch_resident_cycle<double>(const ResidentCycle<double>&, cudaStream_t);
template unsigned prepare_resident<float>(size_t&);
template unsigned prepare_resident<double>(size_t&);

}  // namespace hhg
