// Host-side description of a lattice macro mesh and of its refined levels.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "hhg_common.h"

namespace hhg {

struct BoundaryFace {
  int64_t v[3][3];   // macro lattice coordinates of the three vertices
  uint8_t flag;      // 1 Dirichlet, 2 outflow
  double normal[3];  // outward unit normal
  double area;       // area in physical units
};

struct MacroLattice {
  double origin[3] = {0, 0, 0};
  double H = 1.0;                    // macro cell edge length
  int mx = 0, my = 0, mz = 0;        // macro cells per axis
  std::vector<uint8_t> mask;         // per macro cell: bit s = Kuhn path s present
  std::vector<BoundaryFace> bfaces;  // faces of the macro mesh boundary
  bool has_outflow = false;
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
// its active incident tetrahedra (a 24-bit pattern); all nodes of a class
// have the same assembled rows.  For every class the table holds, in
// doubles and at unit lattice spacing, the 15-point row weights (offset
// order of STENCIL_OFFSETS) of:
//   [W_LAP, +15)   sum_T int grad phi_i . grad phi_j     (A = nu h *, C = delta h_T^2 h *)
//   [W_B + 15 d)   B_d row  -sum_T int phi_i d_d phi_j   (times h^2)
//   [W_BT + 15 d)  B_d^T row                             (times h^2)
//   [W_M, +15)     consistent mass row                   (times h^3)
//   [W_LUMP]       lumped mass int phi_i                 (times h^3)
// cls receives the class of every lattice node (0 for nodes that are not
// F_IRR; classes of F_IRR nodes start at 1), table receives
// (n_classes + 1) * W_STRIDE doubles (class 0 unused).
// Offsets of the 15-point pattern: 0 = centre, 1..7 = +o, 8..14 = -o over the
// Kuhn directions o = e1, e2, e3, e1+e2, e2+e3, e1+e3, e1+e2+e3.
extern const int STENCIL_OFFSETS[15][3];
void stencil_classes(const MacroLattice& m, int level, const uint8_t* flags, std::vector<uint16_t>& cls,
                     std::vector<double>& table, int& n_classes, std::string& err);

}  // namespace hhg
