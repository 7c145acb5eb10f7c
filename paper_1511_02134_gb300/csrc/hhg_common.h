// Lattice description shared by the host mesh builder and the CUDA kernels.
//
// A macro mesh accepted by this library is a set of Kuhn tetrahedra of the
// cells of an axis-aligned lattice of spacing H: tetrahedron "path s" of a
// cell has the vertices  o, o+e_s0, o+e_s0+e_s1, o+(1,1,1)  (o = cell origin).
// Regular (Bey/Freudenthal) refinement of such tetrahedra, level l times,
// yields the Kuhn lattice of spacing h = H / 2^l (Sec. 2.1 uniform
// refinement; each step splits a tetrahedron into 8, Sec. 4).  All levels
// are stored as one node lattice over the bounding box of the macro mesh
// (the union of the paper's vertex/edge/face/volume primitive containers),
// with per-node flags saying which nodes carry velocity / pressure unknowns.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define HHG_HD __host__ __device__ __forceinline__
#else
#define HHG_HD inline
#endif

namespace hhg {

// node flag bits
enum : uint8_t {
  F_ACT = 1,    // node of an active tetrahedron: pressure unknown
  F_VFREE = 2,  // active and not on a Dirichlet face: velocity unknown
  F_IRR = 4,    // some of the 24 incident tetrahedra are inactive (partial stencil)
  F_DIR = 8,    // lies on a Dirichlet face
  F_OUT = 16,   // lies on a do-nothing outflow face
  F_SLIP = 32,  // free velocity node on a free-slip face (always F_IRR)
};

// Padded level arrays: node (i, j, k) of an nx x ny x nz lattice, with a
// ghost frame of one node, has padded coordinates (i+1, j+1, k+1).  Rows
// (px entries, px a multiple of 16) store their entries grouped by padded x
// index q mod 4: entry (q mod 4) px/4 + q div 4.  The nodes of one colour,
// (i + j + k) mod 4 fixed, are then contiguous within each row, so a colour
// sweep reads and writes whole sectors.  Planes hold px * py entries.
HHG_HD int64_t row_pos(int64_t q, int64_t px) { return (q & 3) * (px >> 2) + (q >> 2); }
HHG_HD int64_t pad_index(int64_t px, int64_t pxy, int i, int j, int k) {
  return row_pos(i + 1, px) + px * (j + 1) + pxy * (k + 1);
}
// Row distance from padded x index q to q - 1 and to q + 1.
HHG_HD int64_t row_step_minus(int64_t q, int64_t px) { return (q & 3) == 0 ? 3 * (px >> 2) - 1 : -(px >> 2); }
HHG_HD int64_t row_step_plus(int64_t q, int64_t px) { return (q & 3) == 3 ? 1 - 3 * (px >> 2) : (px >> 2); }

// Layout of one stencil-class row table (unit lattice spacing): stiffness
// row, B_d rows, B_d^T rows, mass row (15 weights each, offset order:
// centre, +o then -o over the Kuhn directions e1, e2, e3, e1+e2, e2+e3,
// e1+e3, e1+e2+e3), lumped mass.
// Classes of free-slip nodes (Sec. 6.1) also hold their constraint: W_SLIP = 1
// with the mass-conservative unit normal <grad phi, 1> / |<grad phi, 1>| at
// W_NRM (velocity in its tangent plane), or W_SLIP = 2 with a unit edge
// direction at W_NRM (two non-parallel free-slip face planes meet at the
// node: velocity along the edge); W_SLIP = 0 for every other class.
constexpr int W_LAP = 0, W_B = 15, W_BT = 60, W_M = 105, W_LUMP = 120, W_NRM = 121, W_SLIP = 124, W_STRIDE = 128;
// Rows of the D-operator velocity block (Sec. 2.1, a_2) of one class (unit
// lattice spacing): block (a, b) = row component a, column component b at
// [15 (3 a + b), +15) in the same offset order, then the inverse of the
// 3 x 3 centre block (row-major) at W2_DINV (for a free-slip class instead
// Z = T (T^T D T)^-1 T^T, T an orthonormal basis of the admissible velocities:
// the node-block update with the slip constraint imposed).  Class 0 holds the rows of the
// nodes with all 24 incident tetrahedra.
constexpr int W2_DINV = 135, W2_STRIDE = 144;

// Kuhn path index of the axis permutation (a, b, c), lexicographic order:
// (0,1,2)=0 (0,2,1)=1 (1,0,2)=2 (1,2,0)=3 (2,0,1)=4 (2,1,0)=5
HHG_HD int path_index(int a, int b, int c) { return 2 * a + (b > c ? 1 : 0); }
HHG_HD int path_axis(int s, int m) {
  // axis of the m-th step (m = 0, 1, 2) of path s
  const int first = s >> 1;
  const int r0 = first == 0 ? 1 : 0;          // smaller remaining axis
  const int r1 = first == 2 ? 1 : 2;          // larger remaining axis
  const int second = (s & 1) ? r1 : r0;
  const int third = 3 - first - second;
  return m == 0 ? first : (m == 1 ? second : third);
}

// Local vertex number (0..3, along the path) of cell corner q = (qx,qy,qz) in
// {0,1}^3 within tetrahedron of path s, or -1 if the corner is not a vertex.
HHG_HD int corner_local(int s, int qx, int qy, int qz) {
  const int n = qx + qy + qz;
  if (n == 0) return 0;
  if (n == 3) return 3;
  const int q[3] = {qx, qy, qz};
  const int a0 = path_axis(s, 0), a1 = path_axis(s, 1);
  if (n == 1) return q[a0] ? 1 : -1;
  return (q[a0] && q[a1]) ? 2 : -1;
}

// Activity of fine tetrahedron (cell c, path s) at refinement level `level`:
// it lies in the macro cell c >> level and inside the macro tetrahedron whose
// path orders the coordinates of its centroid 4c + (3,2,1 along s)
// decreasingly (fine tets of the regular refinement nest in macro tets).
HHG_HD bool tet_active(const uint8_t* macro_mask, int mx, int my, int mz, int level,
                       int cx, int cy, int cz, int s) {
  const int N = 1 << level;
  if (cx < 0 || cy < 0 || cz < 0 || cx >= mx * N || cy >= my * N || cz >= mz * N) return false;
  const int Mx = cx >> level, My = cy >> level, Mz = cz >> level;
  const uint8_t m = macro_mask[Mx + mx * (My + my * Mz)];
  if (m == 0) return false;
  if (m == 63) return true;
  const int q[3] = {cx & (N - 1), cy & (N - 1), cz & (N - 1)};
  int key[3];
  key[path_axis(s, 0)] = 4 * q[path_axis(s, 0)] + 3;
  key[path_axis(s, 1)] = 4 * q[path_axis(s, 1)] + 2;
  key[path_axis(s, 2)] = 4 * q[path_axis(s, 2)] + 1;
  // descending order of keys
  int a = 0, b = 1, c = 2, t;
  if (key[a] < key[b]) { t = a; a = b; b = t; }
  if (key[b] < key[c]) { t = b; b = c; c = t; }
  if (key[a] < key[b]) { t = a; a = b; b = t; }
  return (m >> path_index(a, b, c)) & 1;
}

// Element matrix of int grad(lambda_m).grad(lambda_n) on a Kuhn tetrahedron
// of a unit cell (vertices in path order), times 6:
//   [[1,-1,0,0],[-1,2,-1,0],[0,-1,2,-1],[0,0,-1,1]]
// On a cell of size h the stiffness is h/6 times this.
HHG_HD int kuhn_stiff6(int m, int n) {
  if (m == n) return (m == 0 || m == 3) ? 1 : 2;
  const int d = m - n;
  return (d == 1 || d == -1) ? -1 : 0;
}

}  // namespace hhg
