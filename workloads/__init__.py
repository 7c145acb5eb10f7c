"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds input data only: macro meshes, boundary data, the
manufactured solution and seeded random fields.  It contains none of the
solver's arithmetic (no element integrals, stencils, smoothers or transfers),
so both the CUDA path and the CPU oracle can draw identical inputs from it
without sharing any of the method.

Node order for every nodal array produced here is the lattice order of the
bounding box of the macro mesh at a given refinement level: with
``n_x = nx_cells * 2**level + 1`` (and likewise y, z) node ``(i, j, k)`` sits
at ``origin + (i, j, k) * H / 2**level`` and has flat index
``i + n_x * (j + n_y * k)`` (x fastest).  Nodes of the box that belong to no
macro tetrahedron (obstacles) carry values that the solvers ignore.

Workloads (paper: Sec. 4 serial runs, Sec. 5 TME study, Sec. 6 application):
  * unit cube split into the 6 Kuhn tetrahedra that share the diagonal
    (0,0,0)-(1,1,1) ("6 tetrahedrons", Sec. 4);
  * manufactured smooth solution of Sec. 5 (velocity u, pressure p, forcing f);
  * a 16x4x4 channel of unit cubes with a seeded 10 % of its interior cubes
    removed as no-slip obstacles, inflow on x=0 and do-nothing outflow on
    x=16 -- a synthetic stand-in for the sphere bed of Sec. 6, whose NETGEN
    meshes are not available;
  * free-slip variants (Sec. 6.1): the channel with free-slip obstacles and
    the unit cube with free-slip faces x = 0 and x = 1;
  * the paper's random initial guess (Sec. 3.5): u0 ~ U[0,1],
    p0 ~ U[0, 1/h_min];
  * N(0,1) nodal body forces and random directions for the gradient check.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# Boundary-condition codes per macro face (face f of a tet is the face
# opposite its local vertex f).
BC_AUTO = 0       # interior face, or a boundary face treated as Dirichlet
BC_DIRICHLET = 1  # prescribed velocity
BC_OUTFLOW = 2    # do-nothing (natural) boundary
BC_SLIP = 3       # free slip: no flow through the face, no tangential stress (Sec. 6.1)

# The 6 Kuhn tetrahedra of a unit cell: vertex path 0 -> e_a -> e_a+e_b -> 1.
KUHN_PATHS = list(itertools.permutations(range(3)))


@dataclass
class MacroMesh:
    vertices: np.ndarray   # (nv, 3) float64
    tets: np.ndarray       # (nt, 4) int32, vertex order = refinement order
    bc_flags: np.ndarray   # (nt, 4) uint8, per face opposite local vertex f
    cells: tuple           # (nx, ny, nz) unit cells of the bounding box
    spacing: float         # macro cell edge length H
    origin: np.ndarray     # (3,) float64
    removed: tuple = ()    # removed cells (obstacles), as (i, j, k)
    basis: np.ndarray = None  # (3, 3) lattice axes as columns (None: the identity)

    def lattice_dims(self, level: int) -> tuple:
        n = 1 << level
        return tuple(c * n + 1 for c in self.cells)

    def lattice_coords(self, level: int) -> np.ndarray:
        """(n_nodes, 3) coordinates of the bounding-box lattice, x fastest:
        origin + h basis (i, j, k)."""
        nx, ny, nz = self.lattice_dims(level)
        h = self.spacing / (1 << level)
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
        B = np.eye(3) if self.basis is None else np.asarray(self.basis, float)
        return self.origin[None, :] + (ijk * h) @ B.T


def _box_vertex_id(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def box_of_cubes(nx: int, ny: int, nz: int, removed=(), outflow_x_max: bool = False,
                 slip_sides=(), slip_obstacles: bool = False) -> MacroMesh:
    """Union of nx*ny*nz unit cubes, each split into the 6 Kuhn tetrahedra.

    ``removed`` lists cells (i, j, k) left out (obstacles).  Every boundary
    face is Dirichlet, except the faces on x = nx when ``outflow_x_max``, the
    faces on the box sides named in ``slip_sides`` ("x0", "x1", "y0", "y1",
    "z0", "z1": the planes x = 0, x = nx, ...), which are free slip, and the
    obstacle faces when ``slip_obstacles``.
    """
    removed = tuple(sorted(tuple(int(v) for v in c) for c in removed))
    rset = set(removed)
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    verts = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    ids = _box_vertex_id(gi, gj, gk, nx, ny)
    verts[ids.ravel(), 0] = gi.ravel()
    verts[ids.ravel(), 1] = gj.ravel()
    verts[ids.ravel(), 2] = gk.ravel()
    eye = np.eye(3, dtype=int)
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if (i, j, k) in rset:
                    continue
                for path in KUHN_PATHS:
                    p = np.array([i, j, k])
                    vs = [p.copy()]
                    for a in path:
                        p = p + eye[a]
                        vs.append(p.copy())
                    tets.append([_box_vertex_id(*v, nx, ny) for v in vs])
    tets = np.asarray(tets, dtype=np.int32)
    # boundary faces: faces that occur once
    faces = {}
    for t in range(len(tets)):
        for f in range(4):
            key = tuple(sorted(int(v) for m, v in enumerate(tets[t]) if m != f))
            faces[key] = faces.get(key, 0) + 1
    flags = np.zeros(tets.shape, dtype=np.uint8)
    for t in range(len(tets)):
        for f in range(4):
            fv = [int(v) for m, v in enumerate(tets[t]) if m != f]
            if faces[tuple(sorted(fv))] == 1:
                on_out = outflow_x_max and all(verts[v, 0] == nx for v in fv)
                side = None
                for a, ext in enumerate((nx, ny, nz)):
                    for end, val in ((0, 0), (1, ext)):
                        if all(verts[v, a] == val for v in fv):
                            side = "xyz"[a] + str(end)
                slip = (side in slip_sides) if side is not None else slip_obstacles
                flags[t, f] = BC_OUTFLOW if on_out else (BC_SLIP if slip else BC_DIRICHLET)
    return MacroMesh(vertices=verts, tets=tets, bc_flags=flags, cells=(nx, ny, nz),
                     spacing=1.0, origin=np.zeros(3), removed=removed)


def unit_cube() -> MacroMesh:
    """The unit cube as 6 Kuhn tetrahedra, all boundary faces Dirichlet."""
    return box_of_cubes(1, 1, 1)


SHEAR = np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def sheared_cube() -> MacroMesh:
    """The unit cube's 6 Kuhn tetrahedra under the integer shear x' = x + y:
    a parallelepiped of integer-vertex tetrahedra that are not aligned with
    the coordinate axes (the lattice axes are the columns of SHEAR)."""
    m = box_of_cubes(1, 1, 1)
    m.vertices = m.vertices @ SHEAR.T
    m.basis = SHEAR.copy()
    return m


def channel_obstacles(seed: int = 0, nx: int = 16, ny: int = 4, nz: int = 4, fraction: float = 0.1):
    """Seeded choice of obstacle cubes: ``round(fraction * #interior)`` of the
    cubes that touch no face of the channel box."""
    interior = [(i, j, k) for k in range(1, nz - 1) for j in range(1, ny - 1) for i in range(1, nx - 1)]
    n_remove = int(round(fraction * len(interior)))
    order = np.random.default_rng(seed).permutation(len(interior))
    return tuple(sorted(interior[m] for m in order[:n_remove]))


def obstacle_channel(seed: int = 0, nx: int = 16, ny: int = 4, nz: int = 4, fraction: float = 0.1) -> MacroMesh:
    """16x4x4 channel of unit cubes with seeded obstacles, do-nothing outflow on x = nx."""
    return box_of_cubes(nx, ny, nz, removed=channel_obstacles(seed, nx, ny, nz, fraction), outflow_x_max=True)


def slip_channel(seed: int = 0, nx: int = 16, ny: int = 4, nz: int = 4, fraction: float = 0.1) -> MacroMesh:
    """The obstacle channel with free-slip obstacle faces and no-slip walls:
    the synthetic stand-in for the sphere bed with free-slip spheres of
    Sec. 6 (inflow on x = 0, do-nothing outflow on x = nx)."""
    return box_of_cubes(nx, ny, nz, removed=channel_obstacles(seed, nx, ny, nz, fraction), outflow_x_max=True,
                        slip_obstacles=True)


def slip_cube() -> MacroMesh:
    """The unit cube with free-slip faces x = 0 and x = 1 and Dirichlet faces
    elsewhere (the Dirichlet faces own the shared edges)."""
    return box_of_cubes(1, 1, 1, slip_sides=("x0", "x1"))


def sheared_slip_cube() -> MacroMesh:
    """The slip cube under the shear of sheared_cube: free-slip faces on the
    two tilted planes x = y and x = y + 1."""
    m = slip_cube()
    m.vertices = m.vertices @ SHEAR.T
    m.basis = SHEAR.copy()
    return m


# --- manufactured solution of the TME study (Sec. 5) -----------------------

def manufactured_velocity(x: np.ndarray) -> np.ndarray:
    """u = (-4 cos 4x3, 8 cos 8x1, -2 cos 2x2); returns (n, 3)."""
    return np.stack([-4.0 * np.cos(4.0 * x[:, 2]),
                     8.0 * np.cos(8.0 * x[:, 0]),
                     -2.0 * np.cos(2.0 * x[:, 1])], axis=1)


def manufactured_pressure_tilde(x: np.ndarray) -> np.ndarray:
    return np.sin(4.0 * x[:, 0]) * np.sin(8.0 * x[:, 1]) * np.sin(2.0 * x[:, 2])


def manufactured_pressure_mean_unit_cube() -> float:
    """|Omega|^{-1} <p~, 1> over the unit cube, in closed form."""
    return ((1.0 - np.cos(4.0)) / 4.0) * ((1.0 - np.cos(8.0)) / 8.0) * ((1.0 - np.cos(2.0)) / 2.0)


def manufactured_pressure(x: np.ndarray) -> np.ndarray:
    return manufactured_pressure_tilde(x) - manufactured_pressure_mean_unit_cube()


def manufactured_forcing(x: np.ndarray, nu: float = 1.0) -> np.ndarray:
    """f = -nu * Laplace(u) + grad(p), analytic; returns (n, 3)."""
    s4x, c4x = np.sin(4.0 * x[:, 0]), np.cos(4.0 * x[:, 0])
    s8y, c8y = np.sin(8.0 * x[:, 1]), np.cos(8.0 * x[:, 1])
    s2z, c2z = np.sin(2.0 * x[:, 2]), np.cos(2.0 * x[:, 2])
    lap = np.stack([64.0 * np.cos(4.0 * x[:, 2]),
                    -512.0 * np.cos(8.0 * x[:, 0]),
                    8.0 * np.cos(2.0 * x[:, 1])], axis=1)
    grad_p = np.stack([4.0 * c4x * s8y * s2z, 8.0 * s4x * c8y * s2z, 2.0 * s4x * s8y * c2z], axis=1)
    return -nu * lap + grad_p


def channel_inflow(x: np.ndarray, ny: int = 4, nz: int = 4) -> np.ndarray:
    """Inflow profile of peak 1 on x = 0, zero elsewhere: (n, 3)."""
    y, z = x[:, 1], x[:, 2]
    ux = (y * (ny - y)) * (z * (nz - z)) / ((ny * ny / 4.0) * (nz * nz / 4.0))
    out = np.zeros((x.shape[0], 3))
    on_inflow = np.abs(x[:, 0]) < 1e-12
    out[on_inflow, 0] = ux[on_inflow]
    return out


def outflow_flux_weight(x: np.ndarray, ny: int = 4, nz: int = 4) -> np.ndarray:
    """Nodal weight psi(y, z) = y z / (ny nz) of the weighted outflow flux used for
    the gradient check (the unweighted flux does not depend on the body force)."""
    return x[:, 1] * x[:, 2] / float(ny * nz)


# --- seeded random fields ---------------------------------------------------

def random_initial_guess(n_nodes: int, h_min: float, seed: int = 0):
    """Paper protocol: u0 ~ U[0,1] per component, p0 ~ U[0, 1/h_min]; lattice order."""
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(0.0, 1.0, size=(n_nodes, 3))
    p0 = rng.uniform(0.0, 1.0 / h_min, size=n_nodes)
    return u0, p0


def random_body_force(n_nodes: int, seed: int = 1) -> np.ndarray:
    """N(0,1) nodal body force values, (n_nodes, 3), lattice order."""
    return np.random.default_rng(seed).standard_normal((n_nodes, 3))


def random_directions(n_nodes: int, count: int = 32, seed: int = 2) -> np.ndarray:
    """``count`` N(0,1) perturbation directions of a nodal force, (count, n_nodes, 3)."""
    return np.random.default_rng(seed).standard_normal((count, n_nodes, 3))
