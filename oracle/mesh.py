"""Oracle: uniform refinement of a macro tetrahedral mesh (test infrastructure).

Paper, Sec. 2.1: the hierarchy T_0..T_L is built from the initial mesh T_{-2}
by successive uniform refinement; Sec. 4: each refinement step splits a
tetrahedron into 8.  The paper does not print the split rule.  Reading used
here: Bey's (Freudenthal) regular refinement driven by the vertex order given
for each macro tetrahedron.  With the macro vertices v0..v3 and the affine map
    phi(x) = v0 + x1 (v1 - v0) + x2 (v2 - v1) + x3 (v3 - v2),
the reference simplex K = {1 >= x1 >= x2 >= x3 >= 0} is refined k times into
the N^3 (N = 2^k) Freudenthal simplices {z, z+e_s1, z+e_s1+e_s2, z+1}/N that
lie in K, and phi maps them onto the macro tetrahedron.  For a macro tet
that is a Kuhn tetrahedron of a lattice cell (the unit-cube and channel
workloads), this yields the Kuhn lattice of spacing h = H/N.

Nothing here assumes a lattice: nodes are identified across macro tets by
their exact integer position N*x, which requires integer macro vertices.
Lattice coordinates are only derived afterwards (for the colouring).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

_BC_DIRICHLET_CODES = (0, 1)
_BC_OUTFLOW = 2
_BC_SLIP = 3


@dataclass
class RefinedMesh:
    level: int
    N: int                  # intervals per macro edge
    h: float                # lattice spacing H / N (meaningful for lattice macro meshes)
    xyz: np.ndarray         # (n, 3) node coordinates
    key: np.ndarray         # (n, 3) int64 exact node key N * x (integer)
    tets: np.ndarray        # (nT, 4) node ids of fine tetrahedra
    tet_parent: np.ndarray  # (nT,) macro tet of each fine tet
    on_dirichlet: np.ndarray  # (n,) bool, node lies on a Dirichlet macro face
    on_outflow: np.ndarray    # (n,) bool, node lies on a do-nothing macro face
    outflow_tris: np.ndarray  # (nF, 3) node ids of fine triangles on outflow faces
    outflow_normals: np.ndarray  # (nF, 3) outward unit normals of those triangles
    ijk: np.ndarray = field(default=None)  # (n, 3) lattice coordinates, if a lattice
    on_slip: np.ndarray = field(default=None)  # (n,) bool, free-slip node (on a slip face, on no Dirichlet face)

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def free_velocity(self) -> np.ndarray:
        """Velocity DoFs: every node not on a Dirichlet face (Sec. 2.1, V_l)."""
        return ~self.on_dirichlet

    @property
    def has_outflow(self) -> bool:
        return bool(self.on_outflow.any())


def _reference_points(N: int):
    """Lattice points of N*K in path coordinates, N >= z1 >= z2 >= z3 >= 0."""
    pts = [(a, b, c) for a in range(N + 1) for b in range(a + 1) for c in range(b + 1)]
    pts = np.asarray(pts, dtype=np.int64)
    lut = -np.ones((N + 1, N + 1, N + 1), dtype=np.int64)
    lut[pts[:, 0], pts[:, 1], pts[:, 2]] = np.arange(len(pts))
    return pts, lut


def _reference_simplices(N: int, lut: np.ndarray) -> np.ndarray:
    """The N^3 Freudenthal simplices inside N*K, as local point indices (N^3, 4)."""
    out = []
    eye = np.eye(3, dtype=np.int64)
    z = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij"), -1).reshape(-1, 3)
    for s in itertools.permutations(range(3)):
        v = [z, z + eye[s[0]], z + eye[s[0]] + eye[s[1]], z + 1]
        inside = np.ones(len(z), bool)
        for p in v:
            inside &= (p[:, 0] <= N) & (p[:, 0] >= p[:, 1]) & (p[:, 1] >= p[:, 2]) & (p[:, 2] >= 0)
        idx = np.stack([lut[p[inside, 0], p[inside, 1], p[inside, 2]] for p in v], axis=1)
        out.append(idx)
    simp = np.concatenate(out, axis=0)
    assert simp.shape[0] == N ** 3 and (simp >= 0).all()
    return simp


def refine(vertices, tets, bc_flags, level: int, spacing: float = 1.0, basis=None) -> RefinedMesh:
    """Refine the macro mesh ``level`` times (N = 2**level intervals per macro edge).

    vertices: (nv, 3) integer-valued coordinates; tets: (nt, 4) vertex ids in
    refinement order; bc_flags: (nt, 4) per face opposite local vertex f,
    0 = interior/Dirichlet-by-default, 1 = Dirichlet, 2 = do-nothing outflow,
    3 = free slip (Sec. 6.1; Dirichlet wins on shared edges and corners);
    basis (3, 3): lattice axes as columns when the macro mesh is the affine
    image of a lattice (default: the coordinate axes) -- used only to derive
    the lattice coordinates of the nodes (for the colouring).
    """
    V = np.asarray(vertices, dtype=np.float64)
    T = np.asarray(tets, dtype=np.int64)
    F = np.asarray(bc_flags, dtype=np.int64)
    Vi = np.rint(V).astype(np.int64)
    if not np.allclose(V, Vi, rtol=0, atol=1e-12):
        raise NotImplementedError("oracle refinement keys nodes by N*x and needs integer macro vertices")
    N = 1 << level
    pts, lut = _reference_points(N)
    nloc = len(pts)
    # barycentric numerators (N*lambda) of each reference point
    bary = np.stack([N - pts[:, 0], pts[:, 0] - pts[:, 1], pts[:, 1] - pts[:, 2], pts[:, 2]], axis=1)
    # exact integer positions N*x of all (tet, local point) pairs
    keys = np.einsum("pm,tmc->tpc", bary, Vi[T])  # (nt, nloc, 3)
    flat = keys.reshape(-1, 3)
    uniq, inverse = np.unique(flat, axis=0, return_inverse=True)
    inverse = inverse.reshape(len(T), nloc)
    xyz = uniq.astype(np.float64) / N

    simp = _reference_simplices(N, lut)  # (N^3, 4) local ids
    fine = inverse[:, simp]              # (nt, N^3, 4)
    parent = np.repeat(np.arange(len(T)), N ** 3)
    fine = fine.reshape(-1, 4)

    # boundary macro faces: faces occurring in exactly one macro tet
    face_count = {}
    for t in range(len(T)):
        for f in range(4):
            k = tuple(sorted(int(T[t, m]) for m in range(4) if m != f))
            face_count[k] = face_count.get(k, 0) + 1
    n = len(uniq)
    on_dir = np.zeros(n, bool)
    on_out = np.zeros(n, bool)
    on_slip = np.zeros(n, bool)
    out_tris, out_normals = [], []
    simp_local_faces = [[m for m in range(4) if m != f] for f in range(4)]
    for t in range(len(T)):
        for f in range(4):
            k = tuple(sorted(int(T[t, m]) for m in range(4) if m != f))
            if face_count[k] != 1:
                continue
            on_face = bary[:, f] == 0
            ids = inverse[t, on_face]
            if F[t, f] == _BC_OUTFLOW:
                on_out[ids] = True
                # outward unit normal of the macro face
                a, b, c = (V[T[t, m]] for m in range(4) if m != f)
                nrm = np.cross(b - a, c - a)
                if np.dot(nrm, V[T[t, f]] - a) > 0:
                    nrm = -nrm
                nrm = nrm / np.linalg.norm(nrm)
                # fine triangles of this macro face: faces of fine simplices whose
                # three vertices all lie on the macro face (each occurs once)
                for ff in range(4):
                    tri_local = simp[:, simp_local_faces[ff]]
                    sel = on_face[tri_local].all(axis=1)
                    out_tris.append(inverse[t, tri_local[sel]])
                    out_normals.append(np.repeat(nrm[None], int(sel.sum()), axis=0))
            elif F[t, f] in _BC_DIRICHLET_CODES:
                on_dir[ids] = True
            elif F[t, f] == _BC_SLIP:
                on_slip[ids] = True
            else:
                raise ValueError(f"unknown boundary flag {F[t, f]}")
    if out_tris:
        out_tris = np.concatenate(out_tris, axis=0)
        out_normals = np.concatenate(out_normals, axis=0)
    else:
        out_tris = np.zeros((0, 3), np.int64)
        out_normals = np.zeros((0, 3))

    h = spacing / N
    mesh = RefinedMesh(level=level, N=N, h=h, xyz=xyz, key=uniq, tets=fine, tet_parent=parent,
                       on_dirichlet=on_dir, on_outflow=on_out & ~on_dir,
                       outflow_tris=out_tris, outflow_normals=out_normals, on_slip=on_slip & ~on_dir)
    # lattice coordinates (only meaningful when the macro mesh lives on a lattice of spacing H)
    Binv = np.eye(3) if basis is None else np.linalg.inv(np.asarray(basis, float))
    lat = xyz @ Binv.T
    origin = lat.min(axis=0)
    ijk_f = (lat - origin[None, :]) / h
    ijk = np.rint(ijk_f).astype(np.int64)
    if np.allclose(ijk_f, ijk, rtol=0, atol=1e-9):
        mesh.ijk = ijk
    return mesh


def node_on_outflow_face(mesh: RefinedMesh) -> np.ndarray:
    """Nodes that lie on an outflow face, including its Dirichlet rim."""
    m = np.zeros(mesh.n_nodes, bool)
    if len(mesh.outflow_tris):
        m[mesh.outflow_tris.ravel()] = True
    return m
