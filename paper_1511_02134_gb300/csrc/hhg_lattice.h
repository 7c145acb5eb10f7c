// Host-side description of a lattice macro mesh and of its refined levels.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "hhg_common.h"

namespace hhg {

struct BoundaryFace {
  int64_t v[3][3];   // macro lattice coordinates of the three vertices
  uint8_t flag;      // 1 Dirichlet, 2 outflow, 3 free slip
  double normal[3];  // outward unit normal
  double area;       // area in physical units
};

struct MacroLattice {
  double origin[3] = {0, 0, 0};
  double H = 1.0;                    // macro cell edge length
  // Lattice axes: a lattice point xi (integer at macro vertices) sits at
  // origin + H * basis * xi.  The identity for axis-aligned meshes; for the
  // affine image of a Kuhn lattice (affine = true) the first tetrahedron's
  // edge vectors with H = 1, and every node then takes its class rows.
  double basis[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double basis_inv_t[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};  // basis^-T
  double det = 1.0;                  // |det basis|: volume factor of the lattice cells
  bool affine = false;
  int mx = 0, my = 0, mz = 0;        // macro cells per axis
  std::vector<uint8_t> mask;         // per macro cell: bit s = Kuhn path s present
  std::vector<BoundaryFace> bfaces;  // faces of the macro mesh boundary
  bool has_outflow = false;
  bool has_slip = false;
};

// Validate and convert a macro mesh.  Returns 0 or a negative HHG_E* code
// with a message in err.
int build_macro_lattice(const double* V, int64_t nv, const int32_t* T, int64_t nt,
                        const uint8_t* bc, MacroLattice& out, std::string& err);

struct LevelShape {
  int level;
  int nx, ny, nz;  // lattice nodes per axis
  int64_t n() const { return (int64_t)nx * ny * nz; }
};

LevelShape level_shape(const MacroLattice& m, int level);

// Node flags (F_* bits) of a level in lattice order (x fastest), n bytes.
void classify_nodes(const MacroLattice& m, int level, uint8_t* flags);

// Outflow weights int_{Gamma_out} phi_i n dS, (n, 3) in lattice order.
void outflow_weights(const MacroLattice& m, int level, double* w);

// Number of active incident tetrahedra (0..24) of node (i, j, k) of a level.
int active_incident(const MacroLattice& m, int level, int i, int j, int k);

// Stencil classes of the nodes flagged F_IRR.  A node's class is the set of
// its active incident tetrahedra (a 24-bit pattern) and, in bit 24, whether
// it is a free-slip node (F_SLIP); all nodes of a class have the same
// assembled rows.  For every class the table holds, in
// doubles and at unit lattice spacing, the 15-point row weights (offset
// order of STENCIL_OFFSETS) of:
//   [W_LAP, +15)   sum_T int grad phi_i . grad phi_j     (A = nu h *, C = delta h_T^2 h *)
//   [W_B + 15 d)   B_d row  -sum_T int phi_i d_d phi_j   (times h^2)
//   [W_BT + 15 d)  B_d^T row                             (times h^2)
//   [W_M, +15)     consistent mass row                   (times h^3)
//   [W_LUMP]       lumped mass int phi_i                 (times h^3)
//   [W_NRM, +3)    free-slip classes: unit normal <grad phi_i, 1> / |.|, or
//                  the unit edge direction where two face planes meet
//   [W_SLIP]       1 (normal) or 2 (edge) for free-slip classes
// cls receives the class of every lattice node (0 for nodes that are not
// F_IRR; classes of F_IRR nodes start at 1), table receives
// (n_classes + 1) * W_STRIDE doubles (class 0 unused).
// Offsets of the 15-point pattern: 0 = centre, 1..7 = +o, 8..14 = -o over the
// Kuhn directions o = e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3.
extern const int STENCIL_OFFSETS[15][3];
// patterns (optional) receives the key of each class: the set of active
// incident tetrahedra (bit per (cell corner, Kuhn path) pair; class 0: all
// 24), SLIP_CLASS_BIT for free-slip classes and OUTFLOW_CLASS_BIT for
// free-slip nodes that also lie on an outflow face.
constexpr uint32_t FULL_STAR_PATTERN = (1u << 24) - 1;
constexpr uint32_t SLIP_CLASS_BIT = 1u << 24;
constexpr uint32_t OUTFLOW_CLASS_BIT = 1u << 25;
void stencil_classes(const MacroLattice& m, int level, const uint8_t* flags, std::vector<uint16_t>& cls,
                     std::vector<double>& table, int& n_classes, std::string& err,
                     std::vector<uint32_t>* patterns = nullptr);
// D-operator row tables (W2_STRIDE doubles per class, hhg_common.h) of the
// classes with the given patterns.
void stencil_classes_d(const MacroLattice& m, const std::vector<uint32_t>& patterns, std::vector<double>& table2);

}  // namespace hhg

namespace hhg {

// Compact form of the coarsest level for the coarse solver (Sec. 3.7).  The
// unknowns are numbered component by component over the free velocity nodes
// (lattice order), then over the active pressure nodes (lattice order):
// x = (u_0, u_1, u_2, p), 3 nv + np entries.  K is the saddle-point matrix
// [A 0 0 B_0^T; 0 A 0 B_1^T; 0 0 A B_2^T; B_0 B_1 B_2 -C] and A the scalar
// vector-Laplacian block, both in CSR with the rows of the stencil kernels:
// the class tables for boundary nodes, the closed forms for full-star nodes,
// the same scale factors (A = nu h *, B = h^2 *, C = delta h_T^2 h *).
// Zero weights are not stored.
struct CoarseMatrix {
  int32_t nv = 0, np = 0;
  int32_t coupled = 0;  // D form or free slip: A is the coupled 3 nv x 3 nv velocity block (rows d nv + r)
  std::vector<int32_t> vidx, pidx;  // padded lattice index of each velocity / pressure unknown
  std::vector<int32_t> kptr, kcol;
  std::vector<double> kval;
  std::vector<int32_t> aptr, acol;
  std::vector<double> aval;
  std::vector<double> mass;  // lumped mass of each pressure unknown
};

// flags and cls in lattice order (x fastest); table as from stencil_classes;
// px, pxy the padded strides of the level's fields (ghost frame of one node).
// Returns 0, or HHG_EINVAL when the matrix would not fit 32-bit indices.
// table2 (D form, else null): the D-operator rows per class; the velocity
// block of K and A are then the coupled a_2 rows.  Free-slip nodes (F_SLIP)
// take the velocity block Pi (.) Pi + n n^T and the coupling blocks Pi B^T,
// B Pi (Pi = I - n n^T with the class normal), also in coupled form.
int assemble_coarse(const LevelShape& sh, int64_t px, int64_t pxy, const uint8_t* flags, const uint16_t* cls,
                    const double* table, double nuh, double c, double h2, double h3, CoarseMatrix& out,
                    std::string& err, const double* table2 = nullptr);

}  // namespace hhg
