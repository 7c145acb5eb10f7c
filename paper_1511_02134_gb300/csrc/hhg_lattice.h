// Host-side description of a lattice macro mesh and of its refined levels.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

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

}  // namespace hhg
