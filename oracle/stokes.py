"""Oracle: the discrete Stokes system on one level (test infrastructure).

Builds the block system of Sec. 3 (the linear system with matrix
K = [A B^T; B -C] and right-hand side (f, g); A = A_1 per component in the
Laplace form, the coupled A_2 in the D form, Sec. 2.1) from the assembled operators of
oracle.fem, with the Dirichlet velocity nodes eliminated (Sec. 2.1: the
velocity space carries the boundary condition, the pressure is free at every
node).  Vectors are kept as u: (3, n_u) over the free velocity nodes and
p: (n_p,) over all nodes of the level.

Readings where the paper is silent:
  * right-hand side: the body force enters through its nodal interpolant,
    f_h = M I_h f and g_h = sum_d G_d (I_h f)_d, integrated exactly;
  * inhomogeneous Dirichlet data u_D is lifted: f <- f - A_{I,D} u_D,
    g <- g - B_{.,D} u_D;
  * pure-Dirichlet problems: g is projected onto the range of K by removing
    its Euclidean mean (the null vector of K is (0, 1)), and the pressure is
    normalised by sum_i m_i p_i = 0 (the discrete L^2_0 condition, Sec. 2).

Free slip (Sec. 6.1): u . n_i = 0 at a free-slip node i, with the
mass-conservative normal n_i = <grad phi_i, 1> / |<grad phi_i, 1>| (taken
from B^T 1, whose entries are -<grad phi_i, 1>), and the tangential stress
condition imposed point-wise by testing the momentum rows only in the
tangent plane.  With Pi the projector I - n_i n_i^T at slip nodes (identity
elsewhere) the system solved is
    [Pi A Pi + (I - Pi)   Pi B^T] [u]   [Pi f]
    [B Pi                 -C    ] [p] = [g   ]
whose velocity block is the identity in the normal directions, so their
solution is u . n_i = 0.  Where the free-slip faces at a node are not
coplanar the printed normal is their average; there the node is constrained
by every incident face instead (Pi_i the projector onto the edge direction
where two face planes meet; a corner of three is a Dirichlet node), which
keeps u_i . <grad phi_i, 1> = 0, since that integral lies in the span of the
face normals, and keeps the multigrid contraction independent of the level.
Where <grad phi_i, 1> = 0 (two free-slip faces back to back: obstacles that
touch along an edge or at a corner) there is no normal; such a node is a
contact point of two walls and takes its velocity from the boundary data like
a Dirichlet node (its flux term is zero either way).  Nodes that also lie on
an outflow face keep the printed normal.  Since Pi_i B^T 1 = 0 at slip nodes, the constant
pressure stays in the kernel of a slip-and-Dirichlet problem, and the flux
through slip faces vanishes exactly (the mass-conservation property).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import RefinedMesh, refine


@dataclass
class StokesLevel:
    mesh: RefinedMesh
    ops: fem.Operators
    free: np.ndarray        # indices of free velocity nodes
    dir: np.ndarray         # indices of Dirichlet velocity nodes
    A: sp.csr_matrix        # A restricted to free x free
    A_diag: np.ndarray
    B: list                 # B_d restricted to (all pressure) x free
    BT: list                # transposes
    C: sp.csr_matrix
    C_diag: np.ndarray
    m: np.ndarray           # lumped pressure mass
    pure_dirichlet: bool
    form: str = "laplace"   # "laplace" (a_1) or "D" (a_2, Sec. 2.1)
    A2: sp.csr_matrix = None  # D form: the coupled velocity block over (u_0, u_1, u_2) of the free nodes
    A2_node: np.ndarray = None  # D form: (n_u, 3, 3) diagonal node blocks of A2
    slip: np.ndarray = None     # positions (within free) of the free-slip velocity nodes
    normals: np.ndarray = None  # (n_slip, 3) mass-conservative unit normals of those nodes
    slip_P: np.ndarray = None   # (n_slip, 3, 3) projector onto each node's admissible velocities
    slip_edge: np.ndarray = None  # (n_slip,) bool: constrained by two face planes (velocity along the edge)
    Kv: sp.csr_matrix = None    # coupled velocity block solved (D form or free slip), (u_0, u_1, u_2) order
    Kv_node: np.ndarray = None  # (n_u, 3, 3) diagonal node blocks of Kv

    @property
    def coupled(self) -> bool:
        return self.Kv is not None

    @property
    def n_u(self) -> int:
        return len(self.free)

    @property
    def n_p(self) -> int:
        return self.mesh.n_nodes

    @property
    def n_dofs(self) -> int:
        return 3 * self.n_u + self.n_p

    # --- the operator K and the residual (Sec. 3) --------------------------
    def proj(self, v: np.ndarray) -> np.ndarray:
        """Pi v for v of shape (3, n_u): each slip node's velocity projected on
        its admissible subspace (the tangent plane, or the edge direction)."""
        v = np.array(v, dtype=float, copy=True)
        if self.slip is not None and len(self.slip):
            v[:, self.slip] = np.einsum("nab,bn->an", self.slip_P, v[:, self.slip])
        return v

    def apply_A(self, u: np.ndarray) -> np.ndarray:
        """The velocity block: A u_d per component (Laplace form), or the
        coupled block Kv (D form, free slip)."""
        if self.coupled:
            return (self.Kv @ np.asarray(u).ravel()).reshape(3, self.n_u)
        return np.stack([self.A @ u[d] for d in range(3)])

    def apply(self, u: np.ndarray, p: np.ndarray):
        """K (u, p) = (A u + Pi B^T p,  sum_d B_d (Pi u)_d - C p)."""
        au = self.apply_A(u)
        ru = au + self.proj(np.stack([self.BT[d] @ p for d in range(3)]))
        up = self.proj(u)
        rp = sum(self.B[d] @ up[d] for d in range(3)) - self.C @ p
        return ru, rp

    def residual(self, u, p, f, g):
        """(f, g) - K (u, p)."""
        ku, kp = self.apply(u, p)
        return f - ku, g - kp

    @staticmethod
    def norm(ru, rp) -> float:
        """Euclidean norm over all free DoFs (Sec. 3.6)."""
        return float(np.sqrt(np.sum(ru * ru) + np.sum(rp * rp)))

    def project_pressure(self, p: np.ndarray) -> np.ndarray:
        """Remove the m-weighted mean so that sum_i m_i p_i = 0."""
        if not self.pure_dirichlet:
            return p
        return p - np.dot(self.m, p) / self.m.sum()

    # --- right-hand side ----------------------------------------------------
    def rhs(self, f_nodal=None, u_dirichlet=None):
        """(f, g) for nodal body force f_nodal (n, 3) and boundary data u_dirichlet (n, 3)."""
        n = self.mesh.n_nodes
        fn = np.zeros((n, 3)) if f_nodal is None else np.asarray(f_nodal, float)
        fu = np.stack([(self.ops.M @ fn[:, d])[self.free] for d in range(3)])
        g = sum(self.ops.G[d] @ fn[:, d] for d in range(3))
        if u_dirichlet is not None:
            uD = np.asarray(u_dirichlet, float)
            for d in range(3):
                vd = uD[self.dir, d]
                if self.form == "D":
                    for a in range(3):
                        fu[a] -= self.ops.A2[a][d][self.free][:, self.dir] @ vd
                else:
                    fu[d] -= self.ops.A[self.free][:, self.dir] @ vd
                g = g - self.ops.B[d][:, self.dir] @ vd
        if self.pure_dirichlet:
            g = g - g.mean()
        return self.proj(fu), g

    def scatter(self, u: np.ndarray, u_dirichlet=None) -> np.ndarray:
        """Full nodal velocity (n, 3) from free values (3, n_u) and boundary data."""
        out = np.zeros((self.mesh.n_nodes, 3))
        if u_dirichlet is not None:
            out[self.dir] = np.asarray(u_dirichlet)[self.dir]
        out[self.free] = u.T
        return out


def boundary_face_normal_sums(mesh: RefinedMesh) -> np.ndarray:
    """(n, 3, 3): sum of n_f n_f^T over the boundary faces f of the fine mesh
    incident to each node (n_f the outward unit normal)."""
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = mesh.tets[:, loc].reshape(-1, 3)
    opp = mesh.tets.reshape(-1)
    key = np.sort(faces, axis=1)
    _, first, counts = np.unique(key, axis=0, return_index=True, return_counts=True)
    bnd = first[counts == 1]
    f, o = faces[bnd], opp[bnd]
    X = mesh.xyz
    nrm = np.cross(X[f[:, 1]] - X[f[:, 0]], X[f[:, 2]] - X[f[:, 0]])
    flip = np.sum(nrm * (X[o] - X[f[:, 0]]), axis=1) > 0
    nrm[flip] *= -1.0
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    S = np.zeros((mesh.n_nodes, 3, 3))
    outer = nrm[:, :, None] * nrm[:, None, :]
    for c in range(3):
        np.add.at(S, f[:, c], outer)
    return S


def build_level(mesh: RefinedMesh, nu: float = 1.0, delta: float = 1.0 / 12.0, form: str = "laplace") -> StokesLevel:
    ops = fem.assemble(mesh, nu=nu, delta=delta)
    on_slip = mesh.on_slip if mesh.on_slip is not None else np.zeros(mesh.n_nodes, bool)
    # <grad phi_i, 1> = -(B^T 1)_i, component by component (Sec. 6.1)
    gint_all = -np.stack([ops.B[d].T @ np.ones(mesh.n_nodes) for d in range(3)], axis=1)
    edge_t = np.zeros((mesh.n_nodes, 3))
    is_edge = np.zeros(mesh.n_nodes, bool)
    if on_slip.any():
        pinch = on_slip & (np.linalg.norm(gint_all, axis=1) <= 1e-12 * mesh.h ** 2)
        # rank of the incident face normals at pure slip nodes (not on an outflow face)
        S = boundary_face_normal_sums(mesh)
        cand = np.where(on_slip & ~pinch & ~mesh.on_outflow)[0]
        w, V = np.linalg.eigh(S[cand])
        rank = np.sum(w > 1e-9 * w[:, -1:], axis=1)
        corner = np.zeros(mesh.n_nodes, bool)
        corner[cand[rank >= 3]] = True
        is_edge[cand[rank == 2]] = True
        edge_t[cand[rank == 2]] = V[rank == 2][:, :, 0]   # the null direction of the two face normals
        stop = pinch | corner
        if stop.any():
            mesh.on_dirichlet = mesh.on_dirichlet | stop
            mesh.on_slip = on_slip & ~stop
            on_slip = mesh.on_slip
    free = np.where(mesh.free_velocity)[0]
    dirn = np.where(~mesh.free_velocity)[0]
    A = ops.A[free][:, free].tocsr()
    B = [ops.B[d][:, free].tocsr() for d in range(3)]
    A2, A2_node = None, None
    if form == "D":
        A2 = sp.bmat([[ops.A2[a][b][free][:, free] for b in range(3)] for a in range(3)], format="csr")
        A2_node = np.stack([np.stack([ops.A2[a][b].diagonal()[free] for b in range(3)], axis=1)
                            for a in range(3)], axis=1)
    elif form != "laplace":
        raise ValueError(form)
    L = StokesLevel(mesh=mesh, ops=ops, free=free, dir=dirn, A=A, A_diag=A.diagonal().copy(),
                    B=B, BT=[b.T.tocsr() for b in B], C=ops.C, C_diag=ops.C.diagonal().copy(),
                    m=ops.m, pure_dirichlet=not mesh.has_outflow, form=form, A2=A2, A2_node=A2_node)
    L.slip = np.where(on_slip[free])[0]
    nodes = free[L.slip]
    gint = gint_all[nodes]
    L.normals = gint / np.linalg.norm(gint, axis=1)[:, None] if len(L.slip) else np.zeros((0, 3))
    L.slip_edge = is_edge[nodes]
    t = edge_t[nodes]
    plane = np.eye(3)[None] - L.normals[:, :, None] * L.normals[:, None, :]
    line = t[:, :, None] * t[:, None, :]
    L.slip_P = np.where(L.slip_edge[:, None, None], line, plane)
    couple(L)
    return L


def couple(L: StokesLevel) -> None:
    """Set the coupled velocity block Kv and its node blocks from the form
    and the slip normals: A2 (D form) or A per component (Laplace form),
    constrained as Pi (.) Pi + (I - Pi) at slip nodes.  Nothing to do for the
    Laplace form without slip nodes."""
    if L.form == "D" or len(L.slip):
        n = L.n_u
        blocks = L.A2 if L.form == "D" else sp.block_diag([L.A, L.A, L.A], format="csr")
        if len(L.slip):
            # Pi (A) Pi + (I - Pi), with Pi the slip nodes' projectors (identity elsewhere) as a 3 n x 3 n matrix
            rows, cols, vals = [], [], []
            for a in range(3):
                for b in range(3):
                    rows.append(a * n + L.slip)
                    cols.append(b * n + L.slip)
                    vals.append((1.0 if a == b else 0.0) - L.slip_P[:, a, b])
            Nn = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(3 * n, 3 * n)).tocsr()
            Pi = sp.identity(3 * n, format="csr") - Nn
            blocks = (Pi @ blocks @ Pi + Nn).tocsr()
            blocks.eliminate_zeros()
        L.Kv = blocks
        L.Kv_node = np.stack([np.stack([blocks[a * n:(a + 1) * n, b * n:(b + 1) * n].diagonal() for b in range(3)],
                                       axis=1) for a in range(3)], axis=1)


def build_from_macro(macro, level: int, nu: float = 1.0, delta: float = 1.0 / 12.0,
                     form: str = "laplace") -> StokesLevel:
    mesh = refine(macro.vertices, macro.tets, macro.bc_flags, level, spacing=macro.spacing,
                  basis=getattr(macro, "basis", None))
    return build_level(mesh, nu=nu, delta=delta, form=form)


def full_matrix(L: StokesLevel) -> sp.csr_matrix:
    """K as one sparse matrix, unknown order (u_0, u_1, u_2, p)."""
    Z = [[None] * 4 for _ in range(4)]
    n = L.n_u
    # Pi as 3 x 3 blocks of diagonal matrices over the free nodes
    Pi = [[sp.identity(n, format="csr") if a == b else sp.csr_matrix((n, n)) for b in range(3)] for a in range(3)]
    if len(L.slip):
        for a in range(3):
            for b in range(3):
                dg = np.zeros(n)
                dg[L.slip] = (1.0 if a == b else 0.0) - L.slip_P[:, a, b]
                Pi[a][b] = Pi[a][b] - sp.diags(dg, format="csr")
    for d in range(3):
        if L.coupled:
            for e in range(3):
                Z[d][e] = L.Kv[d * n:(d + 1) * n, e * n:(e + 1) * n]
        else:
            Z[d][d] = L.A
        Z[d][3] = sum(Pi[d][e] @ L.BT[e] for e in range(3))
        Z[3][d] = sum(L.B[e] @ Pi[e][d] for e in range(3))
    Z[3][3] = -L.C
    return sp.bmat(Z, format="csr")
