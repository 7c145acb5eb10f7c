// Host-side lattice logic: macro mesh validation, node classification,
// boundary rasterisation and outflow weights.  Pure C++ (no CUDA), so the
// classification can be checked on machines without a GPU.
#include "hhg_lattice.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <thread>
#include <unordered_map>

#include "../../include/hhg_stokes.h"
#include "hhg_common.h"

namespace hhg {

namespace {

using Key3 = std::array<int64_t, 3>;

int axis_step(const Key3& d, int* sign) {
  // returns the axis if d is +-e_axis, else -1
  int nz = 0, ax = -1;
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0) {
      ++nz;
      ax = a;
    }
  }
  if (nz != 1 || (d[ax] != 1 && d[ax] != -1)) return -1;
  *sign = (int)d[ax];
  return ax;
}

}  // namespace

int build_macro_lattice(const double* V, int64_t nv, const int32_t* T, int64_t nt,
                        const uint8_t* bc, MacroLattice& out, std::string& err) {
  if (!V || !T || nv < 4 || nt < 1) {
    err = "macro mesh needs at least 4 vertices and 1 tetrahedron";
    return HHG_EINVAL;
  }
  for (int64_t t = 0; t < nt * 4; ++t) {
    if (T[t] < 0 || T[t] >= nv) {
      err = "tetrahedron vertex id out of range";
      return HHG_EINVAL;
    }
  }
  // lattice axes from the first tetrahedron: its edges v1 - v0, v2 - v1,
  // v3 - v2; axis-aligned edges of one length give the identity basis with
  // that spacing, anything else the affine lattice of those edge vectors
  double E[3][3];  // E[a][c]: component a of edge c
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) E[a][c] = V[3 * T[c + 1] + a] - V[3 * T[c] + a];
  double len[3];
  bool aligned = true;
  for (int c = 0; c < 3; ++c) {
    len[c] = std::sqrt(E[0][c] * E[0][c] + E[1][c] * E[1][c] + E[2][c] * E[2][c]);
    int nzc = 0;
    for (int a = 0; a < 3; ++a) nzc += E[a][c] != 0.0;
    aligned = aligned && nzc == 1;
  }
  const double H = aligned ? len[0] : 1.0;
  if (!(len[0] > 0) || !std::isfinite(len[0])) {
    err = "degenerate first edge";
    return HHG_EMESH;
  }
  aligned = aligned && std::fabs(len[1] - H) <= 1e-12 * H && std::fabs(len[2] - H) <= 1e-12 * H;
  double Bi[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};  // lattice coordinates per physical unit (x H for aligned)
  if (!aligned) {
    const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                       E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                       E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    if (!(std::fabs(det) > 1e-12 * len[0] * len[1] * len[2]) || !std::isfinite(det)) {
      err = "degenerate first tetrahedron";
      return HHG_EMESH;
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
        Bi[r][c] = (E[r1][c1] * E[r2][c2] - E[r1][c2] * E[r2][c1]) / det;
      }
    out.affine = true;
    out.det = std::fabs(det);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        out.basis[r][c] = E[r][c];
        out.basis_inv_t[r][c] = Bi[c][r];
      }
  }
  // lattice coordinates of the vertices: Bi (v - v0) / H, integers
  const double* v0 = V + 3 * T[0];
  std::vector<std::array<double, 3>> xi(nv);
  double lo[3] = {INFINITY, INFINITY, INFINITY};
  std::vector<char> used(nv, 0);
  for (int64_t t = 0; t < nt * 4; ++t) used[T[t]] = 1;
  for (int64_t v = 0; v < nv; ++v) {
    if (!used[v]) continue;
    for (int a = 0; a < 3; ++a) {
      double x = 0.0;
      for (int c = 0; c < 3; ++c) x += Bi[a][c] * (V[3 * v + c] - v0[c]);
      xi[v][a] = x / H;
      lo[a] = std::min(lo[a], xi[v][a]);
    }
  }
  std::vector<Key3> L(nv, Key3{0, 0, 0});
  for (int64_t v = 0; v < nv; ++v) {
    if (!used[v]) continue;
    for (int a = 0; a < 3; ++a) {
      const double x = xi[v][a] - std::nearbyint(lo[a]);
      const double r = std::nearbyint(x);
      if (!std::isfinite(x) || std::fabs(x - r) > 1e-9 * std::max(1.0, std::fabs(x))) {
        err = "macro vertex not on the lattice of the first tetrahedron's edges";
        return HHG_EMESH;
      }
      L[v][a] = (int64_t)r;
    }
  }
  for (int a = 0; a < 3; ++a) lo[a] = std::nearbyint(lo[a]);
  int64_t hi[3] = {0, 0, 0};
  for (int64_t v = 0; v < nv; ++v)
    if (used[v])
      for (int a = 0; a < 3; ++a) hi[a] = std::max(hi[a], L[v][a]);
  if (hi[0] < 1 || hi[1] < 1 || hi[2] < 1 || hi[0] > 4096 || hi[1] > 4096 || hi[2] > 4096) {
    err = "macro lattice extent out of range";
    return HHG_EMESH;
  }
  out.H = H;
  // physical position of lattice point 0: v0 + H basis lo
  for (int a = 0; a < 3; ++a) {
    double x = v0[a];
    for (int c = 0; c < 3; ++c) x += H * out.basis[a][c] * lo[c];
    out.origin[a] = x;
  }
  out.mx = (int)hi[0];
  out.my = (int)hi[1];
  out.mz = (int)hi[2];
  out.mask.assign((size_t)out.mx * out.my * out.mz, 0);
  out.bfaces.clear();
  out.has_outflow = false;

  // cell and path of every tetrahedron
  for (int64_t t = 0; t < nt; ++t) {
    const Key3& p0 = L[T[4 * t + 0]];
    const Key3& p1 = L[T[4 * t + 1]];
    const Key3& p2 = L[T[4 * t + 2]];
    const Key3& p3 = L[T[4 * t + 3]];
    Key3 d1, d2, d3;
    for (int a = 0; a < 3; ++a) {
      d1[a] = p1[a] - p0[a];
      d2[a] = p2[a] - p1[a];
      d3[a] = p3[a] - p2[a];
    }
    int s1 = 0, s2 = 0, s3 = 0;
    const int a1 = axis_step(d1, &s1), a2 = axis_step(d2, &s2), a3 = axis_step(d3, &s3);
    if (a1 < 0 || a2 < 0 || a3 < 0 || a1 == a2 || a2 == a3 || a1 == a3 || s1 != s2 || s2 != s3) {
      err = "tetrahedron " + std::to_string(t) +
            " is not a lattice Kuhn tetrahedron listed along its path";
      return HHG_EMESH;
    }
    Key3 cell;
    int path;
    if (s1 > 0) {
      cell = p0;
      path = path_index(a1, a2, a3);
    } else {
      cell = p3;
      path = path_index(a3, a2, a1);
    }
    const size_t ci = (size_t)cell[0] + (size_t)out.mx * ((size_t)cell[1] + (size_t)out.my * cell[2]);
    if (out.mask[ci] & (1u << path)) {
      err = "duplicate tetrahedron " + std::to_string(t);
      return HHG_EMESH;
    }
    out.mask[ci] |= (uint8_t)(1u << path);
  }

  // boundary faces: faces that belong to exactly one tetrahedron
  std::map<std::array<int64_t, 9>, std::pair<int, int64_t>> faces;  // key -> (count, t*4+f)
  for (int64_t t = 0; t < nt; ++t) {
    for (int f = 0; f < 4; ++f) {
      std::array<Key3, 3> fv;
      int k = 0;
      for (int m = 0; m < 4; ++m)
        if (m != f) fv[k++] = L[T[4 * t + m]];
      std::sort(fv.begin(), fv.end());
      std::array<int64_t, 9> key;
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) key[3 * i + a] = fv[i][a];
      auto it = faces.find(key);
      if (it == faces.end())
        faces.emplace(key, std::make_pair(1, 4 * t + f));
      else
        it->second.first += 1;
    }
  }
  for (auto& kv : faces) {
    if (kv.second.first > 2) {
      err = "non-manifold macro face";
      return HHG_EMESH;
    }
    if (kv.second.first != 1) continue;
    const int64_t tf = kv.second.second;
    const int64_t t = tf / 4;
    const int f = (int)(tf % 4);
    const uint8_t code = bc ? bc[tf] : (uint8_t)HHG_BC_AUTO;
    if (code > HHG_BC_SLIP) {
      err = "unknown boundary flag";
      return HHG_EINVAL;
    }
    BoundaryFace bf;
    int k = 0;
    for (int m = 0; m < 4; ++m)
      if (m != f) {
        for (int a = 0; a < 3; ++a) bf.v[k][a] = L[T[4 * t + m]][a];
        ++k;
      }
    bf.flag = code == HHG_BC_OUTFLOW ? 2 : (code == HHG_BC_SLIP ? 3 : 1);
    if (bf.flag == 2) out.has_outflow = true;
    if (bf.flag == 3) out.has_slip = true;
    // physical edge vectors of the face (H basis times the lattice differences)
    auto phys = [&](const int64_t* d, double* x) {
      for (int a = 0; a < 3; ++a) {
        x[a] = 0.0;
        for (int c = 0; c < 3; ++c) x[a] += H * out.basis[a][c] * (double)d[c];
      }
    };
    int64_t du[3], dw[3], dq[3];
    for (int a = 0; a < 3; ++a) {
      du[a] = bf.v[1][a] - bf.v[0][a];
      dw[a] = bf.v[2][a] - bf.v[0][a];
      dq[a] = L[T[4 * t + f]][a] - bf.v[0][a];
    }
    double u[3], w[3], q[3], n[3];
    phys(du, u);
    phys(dw, w);
    phys(dq, q);
    n[0] = u[1] * w[2] - u[2] * w[1];
    n[1] = u[2] * w[0] - u[0] * w[2];
    n[2] = u[0] * w[1] - u[1] * w[0];
    const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double to_opp = 0;
    for (int a = 0; a < 3; ++a) to_opp += n[a] * q[a];
    const double sgn = to_opp > 0 ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a) bf.normal[a] = sgn * n[a] / nn;
    bf.area = 0.5 * nn;
    out.bfaces.push_back(bf);
  }
  return HHG_OK;
}

LevelShape level_shape(const MacroLattice& m, int level) {
  LevelShape s;
  s.level = level;
  const int N = 1 << level;
  s.nx = m.mx * N + 1;
  s.ny = m.my * N + 1;
  s.nz = m.mz * N + 1;
  return s;
}

int active_incident(const MacroLattice& m, int level, int i, int j, int k) {
  int count = 0;
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    for (int s = 0; s < 6; ++s) {
      if (corner_local(s, qx, qy, qz) < 0) continue;
      if (tet_active(m.mask.data(), m.mx, m.my, m.mz, level, i - qx, j - qy, k - qz, s)) ++count;
    }
  }
  return count;
}

namespace {

// Visit every fine node of a boundary face at `level`.
template <class F>
void for_face_nodes(const BoundaryFace& bf, int level, F&& fn) {
  const int64_t N = 1ll << level;
  int64_t A[3], U[3], W[3];
  for (int a = 0; a < 3; ++a) {
    A[a] = bf.v[0][a] * N;
    U[a] = bf.v[1][a] - bf.v[0][a];  // one fine step along each macro edge
    W[a] = bf.v[2][a] - bf.v[0][a];
  }
  for (int64_t s = 0; s <= N; ++s)
    for (int64_t t = 0; s + t <= N; ++t)
      fn(A[0] + s * U[0] + t * W[0], A[1] + s * U[1] + t * W[1], A[2] + s * U[2] + t * W[2]);
}

}  // namespace

namespace {
int class_slip_kind(const MacroLattice& mac, uint32_t pattern, double v[3]);

// Set of active incident tetrahedra of node (i, j, k): bit per (cell corner,
// Kuhn path) pair, in the order of the class tables.
uint32_t node_pattern(const MacroLattice& m, int level, int i, int j, int k) {
  uint32_t pattern = 0;
  int bit = 0;
  for (int c = 0; c < 8; ++c) {
    const int qx = c & 1, qy = (c >> 1) & 1, qz = (c >> 2) & 1;
    for (int s = 0; s < 6; ++s) {
      if (corner_local(s, qx, qy, qz) < 0) continue;
      if (tet_active(m.mask.data(), m.mx, m.my, m.mz, level, i - qx, j - qy, k - qz, s)) pattern |= 1u << bit;
      ++bit;
    }
  }
  return pattern;
}
}  // namespace

void classify_nodes(const MacroLattice& m, int level, uint8_t* flags) {
  const LevelShape sh = level_shape(m, level);
  const int N = 1 << level;
  const int64_t nxy = (int64_t)sh.nx * sh.ny;
  auto work = [&](int k0, int k1) {
    for (int k = k0; k < k1; ++k) {
      for (int j = 0; j < sh.ny; ++j) {
        for (int i = 0; i < sh.nx; ++i) {
          int count;
          // fast path: strictly inside one macro cell
          if ((i % N) && (j % N) && (k % N)) {
            const uint8_t mm = m.mask[(size_t)(i / N) + (size_t)m.mx * ((size_t)(j / N) + (size_t)m.my * (k / N))];
            count = mm == 63 ? 24 : (mm == 0 ? 0 : active_incident(m, level, i, j, k));
          } else {
            count = active_incident(m, level, i, j, k);
          }
          uint8_t f = 0;
          if (count > 0) f |= F_ACT;
          // affine lattices: the closed-form rows of the axis-aligned lattice do not apply
          if (count > 0 && (count < 24 || m.affine)) f |= F_IRR;
          flags[i + sh.nx * j + nxy * k] = f;
        }
      }
    }
  };
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if ((int64_t)sh.nx * sh.ny * sh.nz < (1 << 16)) nth = 1;
  std::vector<std::thread> th;
  const int chunk = (sh.nz + (int)nth - 1) / (int)nth;
  for (unsigned t = 0; t < nth; ++t) {
    const int k0 = (int)t * chunk, k1 = std::min(sh.nz, k0 + chunk);
    if (k0 < k1) th.emplace_back(work, k0, k1);
  }
  for (auto& x : th) x.join();
  // boundary faces: Dirichlet, outflow, free slip; a Dirichlet face wins on
  // shared edges and corners
  for (const BoundaryFace& bf : m.bfaces) {
    const uint8_t bit = bf.flag == 1 ? F_DIR : (bf.flag == 2 ? F_OUT : F_SLIP);
    for_face_nodes(bf, level, [&](int64_t x, int64_t y, int64_t z) {
      flags[x + sh.nx * y + nxy * z] |= bit;
    });
  }
  const int64_t n = sh.n();
  for (int64_t i = 0; i < n; ++i) {
    uint8_t f = flags[i];
    if (f & F_DIR) f &= (uint8_t)~(F_OUT | F_SLIP);
    if ((f & F_ACT) && !(f & F_DIR)) f |= F_VFREE;
    if (!(f & F_VFREE)) f &= (uint8_t)~F_SLIP;
    flags[i] = f;
  }
  // A free-slip node whose <grad phi, 1> vanishes (free-slip faces back to
  // back: obstacles touching along an edge or at a corner) has no normal; it
  // is a contact point of two walls.  A node where three free-slip face
  // planes meet (a corner) has no admissible velocity.  Both take their
  // velocity from the boundary data like Dirichlet nodes.
  if (m.has_slip) {
    std::unordered_map<uint32_t, bool> stop;
    for (int k = 0; k < sh.nz; ++k)
      for (int j = 0; j < sh.ny; ++j)
        for (int i = 0; i < sh.nx; ++i) {
          uint8_t& f = flags[i + sh.nx * j + nxy * k];
          if (!(f & F_SLIP)) continue;
          const uint32_t key = node_pattern(m, level, i, j, k) | ((f & F_OUT) ? OUTFLOW_CLASS_BIT : 0u);
          auto it = stop.find(key);
          if (it == stop.end()) {
            double v[3];
            const int kind = class_slip_kind(m, key, v);
            it = stop.emplace(key, kind != 1 && kind != 2).first;
          }
          if (it->second) f = (uint8_t)((f & ~(F_SLIP | F_VFREE)) | F_DIR);
        }
  }
}

const int STENCIL_OFFSETS[15][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {0, 0, 1},  {1, 1, 0},
                                    {0, 1, 1},  {1, 0, 1},  {1, 1, 1},   {-1, 0, 0}, {0, -1, 0},
                                    {0, 0, -1}, {-1, -1, 0}, {0, -1, -1}, {-1, 0, -1}, {-1, -1, -1}};

namespace {

int offset_index(int dx, int dy, int dz) {
  for (int o = 0; o < 15; ++o)
    if (STENCIL_OFFSETS[o][0] == dx && STENCIL_OFFSETS[o][1] == dy && STENCIL_OFFSETS[o][2] == dz) return o;
  return -1;
}

// Rows of one class from the element matrices of its active tetrahedra.
// Tetrahedron (cell corner q of the node, path s) has vertices
// o, o+e_a0, o+e_a0+e_a1, o+(1,1,1) with o = node - q; the unit barycentric
// gradients are g0 = -e_a0, g1 = e_a0 - e_a1, g2 = e_a1 - e_a2, g3 = e_a2;
// |T| = 1/6 at unit spacing.
// Gradients of the barycentric functions in physical directions per lattice
// step: basis^-T g (the identity on axis-aligned lattices); volume factor det.
void geo_grads(const MacroLattice& m, const double g[4][3], double gp[4][3]) {
  for (int n = 0; n < 4; ++n)
    for (int a = 0; a < 3; ++a)
      gp[n][a] = m.basis_inv_t[a][0] * g[n][0] + m.basis_inv_t[a][1] * g[n][1] + m.basis_inv_t[a][2] * g[n][2];
}

// The 24 tetrahedra around a lattice node, in the bit order of a class
// pattern: vertex offsets from the node (lattice steps) along the Kuhn path,
// the node's local index, and for each face containing the node (opposite
// local vertex j != m) the other tetrahedron of the star sharing it.
struct StarTet {
  int v[4][3];
  int m;
  int partner[4];
};

const std::vector<StarTet>& star_tets() {
  static const std::vector<StarTet> star = [] {
    std::vector<StarTet> st;
    for (int q = 0; q < 8; ++q) {
      const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
      for (int s = 0; s < 6; ++s) {
        const int m = corner_local(s, qx, qy, qz);
        if (m < 0) continue;
        StarTet t{};
        t.m = m;
        int p[3] = {0, 0, 0};
        for (int n = 0; n < 4; ++n) {
          if (n > 0) p[path_axis(s, n - 1)] += 1;
          t.v[n][0] = p[0] - qx;
          t.v[n][1] = p[1] - qy;
          t.v[n][2] = p[2] - qz;
        }
        st.push_back(t);
      }
    }
    auto has = [](const StarTet& t, const int* x) {
      for (int n = 0; n < 4; ++n)
        if (t.v[n][0] == x[0] && t.v[n][1] == x[1] && t.v[n][2] == x[2]) return true;
      return false;
    };
    for (size_t a = 0; a < st.size(); ++a)
      for (int j = 0; j < 4; ++j) {
        st[a].partner[j] = -1;
        if (j == st[a].m) continue;
        for (size_t b = 0; b < st.size() && st[a].partner[j] < 0; ++b) {
          if (b == a) continue;
          bool all = true;
          for (int n = 0; n < 4 && all; ++n)
            if (n != j) all = has(st[b], st[a].v[n]);
          if (all) st[a].partner[j] = (int)b;
        }
      }
    return st;
  }();
  return star;
}

// Constraint of a free-slip node from its class key and <grad phi, 1>
// (Sec. 6.1).  1: the unit mass-conservative normal in out (the free-slip
// faces at the node are parallel planes, or the node also lies on an outflow
// face); 2: the unit edge direction in out (the face planes meet in a line:
// velocity along the edge, orthogonal to every face normal and so to
// <grad phi, 1>, which lies in their span); 3: the planes meet in a point
// (corner); 0: the integral vanishes (faces back to back).
int slip_constraint(const MacroLattice& mac, uint32_t key, const double gint[3], double out[3]) {
  const double gn = std::sqrt(gint[0] * gint[0] + gint[1] * gint[1] + gint[2] * gint[2]);
  // the entries are O(1) at unit spacing: a cancellation leaves rounding only
  if (gn <= 1e-12) return 0;
  for (int d = 0; d < 3; ++d) out[d] = gint[d] / gn;
  if (key & OUTFLOW_CLASS_BIT) return 1;
  const std::vector<StarTet>& st = star_tets();
  std::vector<std::array<double, 3>> dirs;
  for (size_t t = 0; t < st.size(); ++t) {
    if (!((key >> t) & 1u)) continue;
    for (int j = 0; j < 4; ++j) {
      if (j == st[t].m) continue;
      const int p = st[t].partner[j];
      if (p >= 0 && ((key >> p) & 1u)) continue;  // face shared with an active tetrahedron
      double x[3][3];
      int c = 0;
      for (int n = 0; n < 4; ++n)
        if (n != j) {
          for (int a = 0; a < 3; ++a)
            x[c][a] = mac.basis[a][0] * st[t].v[n][0] + mac.basis[a][1] * st[t].v[n][1] +
                      mac.basis[a][2] * st[t].v[n][2];
          ++c;
        }
      double e1[3], e2[3], nv[3];
      for (int a = 0; a < 3; ++a) {
        e1[a] = x[1][a] - x[0][a];
        e2[a] = x[2][a] - x[0][a];
      }
      nv[0] = e1[1] * e2[2] - e1[2] * e2[1];
      nv[1] = e1[2] * e2[0] - e1[0] * e2[2];
      nv[2] = e1[0] * e2[1] - e1[1] * e2[0];
      const double l = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      std::array<double, 3> u{nv[0] / l, nv[1] / l, nv[2] / l};
      bool seen = false;
      for (const auto& d : dirs) seen |= std::fabs(d[0] * u[0] + d[1] * u[1] + d[2] * u[2]) > 1.0 - 1e-9;
      if (!seen) dirs.push_back(u);
    }
  }
  if (dirs.size() <= 1) return 1;
  double cvec[3] = {dirs[0][1] * dirs[1][2] - dirs[0][2] * dirs[1][1], dirs[0][2] * dirs[1][0] - dirs[0][0] * dirs[1][2],
                    dirs[0][0] * dirs[1][1] - dirs[0][1] * dirs[1][0]};
  const double cl = std::sqrt(cvec[0] * cvec[0] + cvec[1] * cvec[1] + cvec[2] * cvec[2]);
  for (int a = 0; a < 3; ++a) cvec[a] /= cl;
  for (const auto& d : dirs)
    if (std::fabs(d[0] * cvec[0] + d[1] * cvec[1] + d[2] * cvec[2]) > 1e-9) return 3;
  for (int a = 0; a < 3; ++a) out[a] = cvec[a];
  return 2;
}

void class_rows(const MacroLattice& mac, uint32_t pattern, double* w) {
  std::fill(w, w + W_STRIDE, 0.0);
  const double vol = mac.det;  // 6 |T| at unit lattice spacing
  int bit = 0;
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    for (int s = 0; s < 6; ++s) {
      const int m = corner_local(s, qx, qy, qz);
      if (m < 0) continue;
      const bool active = (pattern >> bit) & 1u;
      ++bit;
      if (!active) continue;
      const int a[3] = {path_axis(s, 0), path_axis(s, 1), path_axis(s, 2)};
      int vx[4][3];
      int p[3] = {0, 0, 0};
      for (int n = 0; n < 4; ++n) {
        if (n > 0) p[a[n - 1]] += 1;
        vx[n][0] = p[0] - qx;
        vx[n][1] = p[1] - qy;
        vx[n][2] = p[2] - qz;
      }
      int idx[4];
      for (int n = 0; n < 4; ++n) idx[n] = offset_index(vx[n][0], vx[n][1], vx[n][2]);
      double g[4][3] = {};
      g[0][a[0]] = -1;
      g[1][a[0]] += 1;
      g[1][a[1]] -= 1;
      g[2][a[1]] += 1;
      g[2][a[2]] -= 1;
      g[3][a[2]] = 1;
      double gp[4][3];
      geo_grads(mac, g, gp);
      for (int n = 0; n < 4; ++n) {
        w[W_LAP + idx[n]] += vol * (gp[m][0] * gp[n][0] + gp[m][1] * gp[n][1] + gp[m][2] * gp[n][2]) / 6.0;
        for (int d = 0; d < 3; ++d) {
          w[W_B + 15 * d + idx[n]] += -vol * gp[n][d] / 24.0;
          w[W_BT + 15 * d + idx[n]] += -vol * gp[m][d] / 24.0;
        }
        w[W_M + idx[n]] += vol / 120.0;
      }
      w[W_M + 0] += vol / 120.0;
      w[W_LUMP] += vol / 24.0;
    }
  }
  if (pattern & SLIP_CLASS_BIT) {
    // <grad phi, 1> = -(B^T 1): minus the sum of the B^T row weights
    double n[3];
    for (int d = 0; d < 3; ++d) {
      n[d] = 0.0;
      for (int o = 0; o < 15; ++o) n[d] -= w[W_BT + 15 * d + o];
    }
    double v[3];
    const int kind = slip_constraint(mac, pattern, n, v);
    for (int d = 0; d < 3; ++d) w[W_NRM + d] = kind == 1 || kind == 2 ? v[d] : 0.0;
    w[W_SLIP] = kind == 1 || kind == 2 ? (double)kind : 0.0;
  }
}

// Constraint kind of a free-slip class (slip_constraint) and its vector.
int class_slip_kind(const MacroLattice& mac, uint32_t pattern, double v[3]) {
  std::vector<double> w(W_STRIDE);
  class_rows(mac, pattern | SLIP_CLASS_BIT, w.data());
  for (int d = 0; d < 3; ++d) v[d] = w[W_NRM + d];
  if (w[W_SLIP] != 0.0) return (int)w[W_SLIP];
  // no stored constraint: contact point (zero integral) or corner
  double n[3];
  for (int d = 0; d < 3; ++d) {
    n[d] = 0.0;
    for (int o = 0; o < 15; ++o) n[d] -= w[W_BT + 15 * d + o];
  }
  double u[3];
  return slip_constraint(mac, pattern | SLIP_CLASS_BIT, n, u);
}

// D-operator rows of one class: per active tetrahedron, with the centre the
// local vertex m and neighbour n, a_2(phi_n e_b, phi_m e_a) =
// nu int (delta_ab grad l_m . grad l_n + d_b l_m d_a l_n) = nu |T| (delta_ab
// g_m . g_n + g_m[b] g_n[a]), |T| = 1/6 at unit spacing; then the centre
// block's inverse.
void class_rows_d(const MacroLattice& mac, uint32_t pattern, double* w) {
  std::fill(w, w + W2_STRIDE, 0.0);
  const double vol = mac.det;
  int bit = 0;
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    for (int s = 0; s < 6; ++s) {
      const int m = corner_local(s, qx, qy, qz);
      if (m < 0) continue;
      const bool active = (pattern >> bit) & 1u;
      ++bit;
      if (!active) continue;
      const int a[3] = {path_axis(s, 0), path_axis(s, 1), path_axis(s, 2)};
      int idx[4];
      int p[3] = {0, 0, 0};
      for (int n = 0; n < 4; ++n) {
        if (n > 0) p[a[n - 1]] += 1;
        idx[n] = offset_index(p[0] - qx, p[1] - qy, p[2] - qz);
      }
      double g[4][3] = {};
      g[0][a[0]] = -1;
      g[1][a[0]] += 1;
      g[1][a[1]] -= 1;
      g[2][a[1]] += 1;
      g[2][a[2]] -= 1;
      g[3][a[2]] = 1;
      double gp[4][3];
      geo_grads(mac, g, gp);
      for (int n = 0; n < 4; ++n) {
        const double gg = gp[m][0] * gp[n][0] + gp[m][1] * gp[n][1] + gp[m][2] * gp[n][2];
        for (int ra = 0; ra < 3; ++ra)
          for (int cb = 0; cb < 3; ++cb)
            w[15 * (3 * ra + cb) + idx[n]] += vol * ((ra == cb ? gg : 0.0) + gp[m][cb] * gp[n][ra]) / 6.0;
      }
    }
  }
  // inverse of the centre block by cofactors (it is symmetric positive definite
  // whenever the node has an active tetrahedron)
  double D[3][3];
  for (int ra = 0; ra < 3; ++ra)
    for (int cb = 0; cb < 3; ++cb) D[ra][cb] = w[15 * (3 * ra + cb)];
  const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                     D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                     D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
  if (det == 0.0) return;
  for (int ra = 0; ra < 3; ++ra)
    for (int cb = 0; cb < 3; ++cb) {
      const int r1 = (cb + 1) % 3, r2 = (cb + 2) % 3, c1 = (ra + 1) % 3, c2 = (ra + 2) % 3;
      w[W2_DINV + 3 * ra + cb] = (D[r1][c1] * D[r2][c2] - D[r1][c2] * D[r2][c1]) / det;
    }
  if (!(pattern & SLIP_CLASS_BIT)) return;
  double n[3];
  const int kind = class_slip_kind(mac, pattern, n);
  if (kind == 2) {
    // along the edge direction t: Z = t t^T / (t^T D t)
    double q = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) q += n[a] * D[a][b] * n[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) w[W2_DINV + 3 * a + b] = n[a] * n[b] / q;
    return;
  }
  if (kind != 1) return;  // contact points and corners are Dirichlet nodes
  // orthonormal tangent basis t1, t2: t1 from the axis least aligned with n
  int e = 0;
  for (int a = 1; a < 3; ++a)
    if (std::fabs(n[a]) < std::fabs(n[e])) e = a;
  double t1[3] = {0, 0, 0}, t2[3];
  t1[e] = 1.0;
  const double dn = n[e];
  for (int a = 0; a < 3; ++a) t1[a] -= dn * n[a];
  const double l1 = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int a = 0; a < 3; ++a) t1[a] /= l1;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
  const double* T[2] = {t1, t2};
  // M = T^T D T (2 x 2), Z = T M^-1 T^T
  double M[2][2];
  for (int x = 0; x < 2; ++x)
    for (int y = 0; y < 2; ++y) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += T[x][a] * D[a][b] * T[y][b];
      M[x][y] = s;
    }
  const double dm = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  const double Mi[2][2] = {{M[1][1] / dm, -M[0][1] / dm}, {-M[1][0] / dm, M[0][0] / dm}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) s += T[x][a] * Mi[x][y] * T[y][b];
      w[W2_DINV + 3 * a + b] = s;
    }
}

}  // namespace

void stencil_classes_d(const MacroLattice& m, const std::vector<uint32_t>& patterns, std::vector<double>& table2) {
  table2.assign(patterns.size() * W2_STRIDE, 0.0);
  for (size_t c = 0; c < patterns.size(); ++c) class_rows_d(m, patterns[c], table2.data() + c * W2_STRIDE);
}

void stencil_classes(const MacroLattice& m, int level, const uint8_t* flags, std::vector<uint16_t>& cls,
                     std::vector<double>& table, int& n_classes, std::string& err, std::vector<uint32_t>* patterns) {
  const LevelShape sh = level_shape(m, level);
  cls.assign((size_t)sh.n(), 0);
  table.assign(W_STRIDE, 0.0);  // class 0: regular nodes (rows not stored)
  std::unordered_map<uint32_t, uint16_t> ids;
  n_classes = 0;
  if (patterns) patterns->assign(1, FULL_STAR_PATTERN);
  for (int k = 0; k < sh.nz; ++k)
    for (int j = 0; j < sh.ny; ++j)
      for (int i = 0; i < sh.nx; ++i) {
        const int64_t q = i + (int64_t)sh.nx * (j + (int64_t)sh.ny * k);
        if (!(flags[q] & F_IRR)) continue;
        const uint32_t pattern = node_pattern(m, level, i, j, k) | ((flags[q] & F_SLIP) ? SLIP_CLASS_BIT : 0u) |
                                 ((flags[q] & F_SLIP) && (flags[q] & F_OUT) ? OUTFLOW_CLASS_BIT : 0u);
        auto it = ids.find(pattern);
        if (it == ids.end()) {
          if (n_classes >= 65535) {
            err = "more than 65535 boundary stencil classes";
            return;
          }
          ++n_classes;
          it = ids.emplace(pattern, (uint16_t)n_classes).first;
          table.resize((size_t)(n_classes + 1) * W_STRIDE);
          class_rows(m, pattern, table.data() + (size_t)n_classes * W_STRIDE);
          if (patterns) patterns->push_back(pattern);
        }
        cls[q] = it->second;
      }
}

void outflow_weights(const MacroLattice& m, int level, double* w) {
  const LevelShape sh = level_shape(m, level);
  const int64_t nxy = (int64_t)sh.nx * sh.ny;
  std::fill(w, w + 3 * sh.n(), 0.0);
  const int64_t N = 1ll << level;
  for (const BoundaryFace& bf : m.bfaces) {
    if (bf.flag != 2) continue;
    // uniform subdivision of the macro triangle into N^2 triangles of equal area
    const double third = bf.area / (double)(N * N) / 3.0;
    int64_t A[3], U[3], W[3];
    for (int a = 0; a < 3; ++a) {
      A[a] = bf.v[0][a] * N;
      U[a] = bf.v[1][a] - bf.v[0][a];
      W[a] = bf.v[2][a] - bf.v[0][a];
    }
    auto node = [&](int64_t s, int64_t t) {
      return (A[0] + s * U[0] + t * W[0]) + sh.nx * (A[1] + s * U[1] + t * W[1]) + nxy * (A[2] + s * U[2] + t * W[2]);
    };
    auto add = [&](int64_t id) {
      for (int a = 0; a < 3; ++a) w[3 * id + a] += third * bf.normal[a];
    };
    for (int64_t s = 0; s < N; ++s) {
      for (int64_t t = 0; s + t < N; ++t) {
        add(node(s, t));
        add(node(s + 1, t));
        add(node(s, t + 1));
        if (s + t + 1 < N) {
          add(node(s + 1, t));
          add(node(s, t + 1));
          add(node(s + 1, t + 1));
        }
      }
    }
  }
}

}  // namespace hhg
