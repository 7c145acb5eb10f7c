// Host assembly of the coarsest-level saddle-point matrix in CSR (Sec. 3.7
// coarse solver; rows of Sec. 2 on the Kuhn lattice).  Full-star nodes take
// the closed-form rows the stencil kernels apply: the 7-point Laplacian
// (6 at the centre, -1 on the six axis neighbours) and B_d = h^2/12 times
// the antisymmetric difference weights along the seven Kuhn directions;
// boundary nodes take their class rows.
#include <limits>

#include "../../include/hhg_stokes.h"
#include "hhg_lattice.h"

namespace hhg {

namespace {

// 12 * (B_d row) on the "+o" neighbour along direction q of
// (e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3); the "-o" neighbour takes the
// opposite sign and the centre weight is zero.
const double DIV12[3][7] = {{-3, 1, 1, -1, 1, -1, -1}, {1, -3, 1, -1, -1, 1, -1}, {1, 1, -3, 1, -1, -1, -1}};

struct Rows {
  double lap[15], b[3][15], bt[3][15], lump;
};

Rows rows_of(uint16_t cls, const double* table) {
  Rows r{};
  if (cls == 0) {
    r.lap[0] = 6.0;
    for (int o : {1, 2, 3, 8, 9, 10}) r.lap[o] = -1.0;
    for (int d = 0; d < 3; ++d)
      for (int q = 0; q < 7; ++q) {
        r.b[d][1 + q] = DIV12[d][q] / 12.0;
        r.b[d][8 + q] = -DIV12[d][q] / 12.0;
        r.bt[d][1 + q] = -DIV12[d][q] / 12.0;
        r.bt[d][8 + q] = DIV12[d][q] / 12.0;
      }
    r.lump = 1.0;
    return r;
  }
  const double* w = table + (size_t)cls * W_STRIDE;
  for (int o = 0; o < 15; ++o) {
    r.lap[o] = w[W_LAP + o];
    for (int d = 0; d < 3; ++d) {
      r.b[d][o] = w[W_B + 15 * d + o];
      r.bt[d][o] = w[W_BT + 15 * d + o];
    }
  }
  r.lump = w[W_LUMP];
  return r;
}

}  // namespace

int assemble_coarse(const LevelShape& sh, int64_t px, int64_t pxy, const uint8_t* flags, const uint16_t* cls,
                    const double* table, double nuh, double c, double h2, double h3, CoarseMatrix& out,
                    std::string& err, const double* table2) {
  out = CoarseMatrix{};
  const int64_t n = sh.n();
  const int64_t nalloc = pxy * (sh.nz + 2);
  if (nalloc > std::numeric_limits<int32_t>::max() / 2) {
    err = "coarsest level too large for the assembled coarse solver";
    return HHG_EINVAL;
  }
  std::vector<int32_t> iv(nalloc, -1), ip(nalloc, -1);
  std::vector<int64_t> lat_of(nalloc, -1);
  std::vector<int32_t> vi, vj, vk, qi, qj, qk;  // lattice coordinates of the unknowns' nodes
  for (int k = 0; k < sh.nz; ++k)
    for (int j = 0; j < sh.ny; ++j)
      for (int i = 0; i < sh.nx; ++i) {
        const int64_t q = i + (int64_t)sh.nx * (j + (int64_t)sh.ny * k);
        const int64_t pc = pad_index(px, pxy, i, j, k);
        lat_of[pc] = q;
        if (flags[q] & F_VFREE) {
          iv[pc] = out.nv++;
          out.vidx.push_back((int32_t)pc);
          vi.push_back(i);
          vj.push_back(j);
          vk.push_back(k);
        }
        if (flags[q] & F_ACT) {
          ip[pc] = out.np++;
          out.pidx.push_back((int32_t)pc);
          qi.push_back(i);
          qj.push_back(j);
          qk.push_back(k);
        }
      }
  (void)n;
  // padded index of the neighbour along stencil offset o (the ghost frame
  // holds the neighbours of boundary nodes; they carry no unknown)
  auto nbr = [&](int i, int j, int k, int o) {
    return pad_index(px, pxy, i + STENCIL_OFFSETS[o][0], j + STENCIL_OFFSETS[o][1], k + STENCIL_OFFSETS[o][2]);
  };
  const int32_t nv = out.nv, np = out.np;
  int64_t nnz = 0;
  auto push = [&](std::vector<int32_t>& col, std::vector<double>& val, int64_t j, double v) {
    if (v == 0.0) return;
    col.push_back((int32_t)j);
    val.push_back(v);
    ++nnz;
  };
  // Free slip (Sec. 6.1): the class row of a slip node (its constraint at
  // W_NRM, W_SLIP), or null; the velocity block is then Pi (.) Pi + (I - Pi)
  // at slip nodes, Pi = I - n n^T (tangent plane) or t t^T (edge direction),
  // and the coupling blocks Pi B^T and B Pi, which couples the components,
  // so the system is assembled in coupled form.
  bool slip = false;
  for (int32_t r = 0; r < nv && !slip; ++r) slip = (flags[lat_of[out.vidx[r]]] & F_SLIP) != 0;
  auto normal_of = [&](int64_t pc) -> const double* {
    const int64_t q = lat_of[pc];
    if (!(flags[q] & F_SLIP)) return nullptr;
    return table + (size_t)cls[q] * W_STRIDE;
  };
  auto pi = [](const double* w, int a, int b) {
    const double id = a == b ? 1.0 : 0.0;
    if (!w || w[W_SLIP] == 0.0) return id;
    const double* v = w + W_NRM;
    return w[W_SLIP] == 1.0 ? id - v[a] * v[b] : v[a] * v[b];
  };
  const bool coupled = table2 != nullptr || slip;
  // 3 x 3 velocity block of row node r and its neighbour along offset o
  auto vblock = [&](int32_t r, const Rows& w, const double* w2, int o, int64_t nb, double V[3][3]) {
    double base[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        base[a][b] = w2 ? nuh * w2[15 * (3 * a + b) + o] : (a == b ? nuh * w.lap[o] : 0.0);
    const double* nr = normal_of(out.vidx[r]);
    const double* nn = normal_of(nb);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int x = 0; x < 3; ++x)
          for (int y = 0; y < 3; ++y) s += pi(nr, a, x) * base[x][y] * pi(nn, y, b);
        V[a][b] = s + (o == 0 && nr ? (a == b ? 1.0 : 0.0) - pi(nr, a, b) : 0.0);
      }
  };
  // velocity rows, component by component
  out.kptr.push_back(0);
  for (int d = 0; d < 3; ++d)
    for (int32_t r = 0; r < nv; ++r) {
      const int64_t pc = out.vidx[r];
      const uint16_t cl = cls[lat_of[pc]];
      const Rows w = rows_of(cl, table);
      const double* w2 = table2 ? table2 + (size_t)cl * W2_STRIDE : nullptr;
      const double* nr = normal_of(pc);
      if (coupled) {
        for (int b = 0; b < 3; ++b)
          for (int o = 0; o < 15; ++o) {
            const int64_t nb = nbr(vi[r], vj[r], vk[r], o);
            if (iv[nb] < 0) continue;
            double V[3][3];
            vblock(r, w, w2, o, nb, V);
            push(out.kcol, out.kval, (int64_t)b * nv + iv[nb], V[d][b]);
          }
      } else {
        for (int o = 0; o < 15; ++o) {
          const int64_t nb = nbr(vi[r], vj[r], vk[r], o);
          if (iv[nb] >= 0) push(out.kcol, out.kval, (int64_t)d * nv + iv[nb], nuh * w.lap[o]);
        }
      }
      for (int o = 0; o < 15; ++o) {
        const int64_t nb = nbr(vi[r], vj[r], vk[r], o);
        if (ip[nb] < 0) continue;
        double v = 0.0;
        for (int e = 0; e < 3; ++e) v += pi(nr, d, e) * h2 * w.bt[e][o];
        push(out.kcol, out.kval, 3 * (int64_t)nv + ip[nb], v);
      }
      if (nnz > std::numeric_limits<int32_t>::max() / 2) {
        err = "coarsest level too large for the assembled coarse solver";
        return HHG_EINVAL;
      }
      out.kptr.push_back((int32_t)nnz);
    }
  // pressure rows: B Pi u - C p
  for (int32_t r = 0; r < np; ++r) {
    const int64_t pc = out.pidx[r];
    const Rows w = rows_of(cls[lat_of[pc]], table);
    for (int d = 0; d < 3; ++d)
      for (int o = 0; o < 15; ++o) {
        const int64_t nb = nbr(qi[r], qj[r], qk[r], o);
        if (iv[nb] < 0) continue;
        const double* nn = normal_of(nb);
        double v = 0.0;
        for (int e = 0; e < 3; ++e) v += h2 * w.b[e][o] * pi(nn, e, d);
        push(out.kcol, out.kval, (int64_t)d * nv + iv[nb], v);
      }
    for (int o = 0; o < 15; ++o) {
      const int64_t nb = nbr(qi[r], qj[r], qk[r], o);
      if (ip[nb] >= 0) push(out.kcol, out.kval, 3 * (int64_t)nv + ip[nb], -c * w.lap[o]);
    }
    if (nnz > std::numeric_limits<int32_t>::max() / 2) {
      err = "coarsest level too large for the assembled coarse solver";
      return HHG_EINVAL;
    }
    out.kptr.push_back((int32_t)nnz);
    out.mass.push_back(h3 * w.lump);
  }
  // A: the coupled block (3 nv rows: D form, free slip), or the scalar Laplacian
  nnz = 0;
  out.aptr.push_back(0);
  if (coupled) {
    out.coupled = 1;
    for (int d = 0; d < 3; ++d)
      for (int32_t r = 0; r < nv; ++r) {
        const uint16_t cl = cls[lat_of[out.vidx[r]]];
        const Rows w = rows_of(cl, table);
        const double* w2 = table2 ? table2 + (size_t)cl * W2_STRIDE : nullptr;
        for (int b = 0; b < 3; ++b)
          for (int o = 0; o < 15; ++o) {
            const int64_t nb = nbr(vi[r], vj[r], vk[r], o);
            if (iv[nb] < 0) continue;
            double V[3][3];
            vblock(r, w, w2, o, nb, V);
            push(out.acol, out.aval, (int64_t)b * nv + iv[nb], V[d][b]);
          }
        out.aptr.push_back((int32_t)nnz);
      }
    return HHG_OK;
  }
  for (int32_t r = 0; r < nv; ++r) {
    const int64_t pc = out.vidx[r];
    const Rows w = rows_of(cls[lat_of[pc]], table);
    for (int o = 0; o < 15; ++o) {
      const int64_t nb = nbr(vi[r], vj[r], vk[r], o);
      if (iv[nb] >= 0) push(out.acol, out.aval, iv[nb], nuh * w.lap[o]);
    }
    out.aptr.push_back((int32_t)nnz);
  }
  return HHG_OK;
}

}  // namespace hhg
