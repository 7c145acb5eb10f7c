"""Oracle: all-at-once Uzawa multigrid, V_var(3,3) (test infrastructure).

Follows the paper's best solver (UMG, Tab. "settings" of Sec. 3.7):
  * inexact Uzawa smoother (Sec. 3.3):
        u_{k+1} = u_k + A_hat^{-1} (f - A u_k - B^T p_k)
        p_{k+1} = p_k + S_hat^{-1} (B u_{k+1} - C p_k - g)
    with A_hat = one forward plus one backward Gauss-Seidel sweep on A
    (the pseudo-symmetric SHGS of Sec. 3.4, both sweeps on the same right-hand
    side f - B^T p_k) and S_hat = one forward Gauss-Seidel sweep on C with
    under-relaxation omega = 0.3 (Sec. 3.5), started from zero, which is the
    in-place update p_i <- p_i + omega (B u - g - C p)_i / C_ii;
  * variable V-cycle: nu_l = 3 + 2 (L - l) pre- and post-smoothing steps on
    level l (Sec. 3.5), residual, restriction, recursion, prolongation;
  * coarsest level: block-preconditioned MINRES (oracle.krylov, Sec. 3.7),
    CG on the velocity block (per component for A_1, on the coupled A_2 in the
    D form) and the lumped mass on the pressure;
  * outer loop: stop when ||K x_k - f~|| / ||K x_0 - f~|| <= eps (Sec. 3.6);
    pure-Dirichlet problems project the pressure to sum m_i p_i = 0 after
    every cycle (K (0, 1) = 0, so the residual is unaffected).

Readings where the paper is silent (the paper's hybrid HHG ordering cannot
be reproduced without its source):
  * Gauss-Seidel order: 4 colours c = (i + j + k) mod 4 in lattice
    coordinates; forward = colours 0,1,2,3, backward = 3,2,1,0.  Nodes of one
    colour are not coupled (checked by colouring_is_valid), so updating a
    colour at once equals any sequential order within it;
  * transfers: P = P1 interpolation from level l-1 to level l (new nodes are
    midpoints of coarse edges and take the mean of its two end values),
    R = P^T, for velocity and pressure alike; the velocity transfers act on
    free nodes only (a coarse Dirichlet node carries no correction);
  * coarse operators are rediscretised on every level (c_l is level
    dependent, Sec. 2.1), not Galerkin products;
  * free slip (Sec. 6.1, oracle.stokes): the smoother works on the coupled
    velocity block Pi A Pi + (I - Pi) with its 3 x 3 node blocks (the update
    of a slip node is the tangential part of its unconstrained update); the
    restricted residual is projected with the coarse normals and the
    prolongated correction with the fine normals, so every level's iterate
    stays tangential at its own slip nodes.

Parity unpinned: h_norm restates the mesh-dependent norm printed in Sec. 5
and serves the reported gamma_l only; no pin distinguishes its weight h^2
on the pressure from another power of h.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import krylov
from .mesh import refine
from .stokes import StokesLevel, build_level


@dataclass
class Options:
    nu_pre: int = 3            # V_var(3,3)
    nu_post: int = 3
    var_increment: int = 2     # two more steps per coarser level
    omega: float = 0.3         # pressure under-relaxation
    coarse_minres_max: int = 5
    coarse_minres_rtol: float = 5e-3
    coarse_cg_max: int = 50
    coarse_cg_rtol: float = 1e-3


def colour_of(L: StokesLevel) -> np.ndarray:
    if L.mesh.ijk is None:
        raise NotImplementedError("4-colouring is defined for lattice meshes")
    return L.mesh.ijk.sum(axis=1) % 4


def colouring_is_valid(L: StokesLevel) -> bool:
    """No non-zero off-diagonal entry of A, C or of the node graph of the mesh
    (the full 15-point pattern) joins two nodes of the same colour."""
    col = colour_of(L)
    tets = L.mesh.tets
    for a in range(4):
        for b in range(a + 1, 4):
            if np.any(col[tets[:, a]] == col[tets[:, b]]):
                return False
    for Mx, rows_cols in ((L.ops.A, None), (L.ops.C, None)):
        coo = Mx.tocoo()
        off = (coo.row != coo.col) & (coo.data != 0)
        if np.any(col[coo.row[off]] == col[coo.col[off]]):
            return False
    return True


def prolongation(fine: StokesLevel, coarse: StokesLevel) -> sp.csr_matrix:
    """P1 interpolation (n_fine x n_coarse) over all nodes, built from coarse edges."""
    kf = fine.mesh.key            # N_f * x
    kc = coarse.mesh.key * 2      # coarse nodes expressed at the fine scale
    lo = np.minimum(kf.min(0), kc.min(0))
    span = np.maximum(kf.max(0), kc.max(0)) - lo + 1

    def pack(k):
        k = k - lo
        return k[:, 0] + span[0] * (k[:, 1] + span[1] * k[:, 2])

    fk = pack(kf)
    order = np.argsort(fk)
    fk_sorted = fk[order]

    def lookup(k):
        pos = np.searchsorted(fk_sorted, pack(k))
        assert np.all(fk_sorted[pos] == pack(k)), "node missing in fine mesh"
        return order[pos]

    rows, cols, vals = [], [], []
    # fine nodes that coincide with coarse nodes
    fc = lookup(kc)
    rows.append(fc)
    cols.append(np.arange(len(kc)))
    vals.append(np.ones(len(kc)))
    # midpoints of coarse edges
    t = coarse.mesh.tets
    edges = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    edges = np.unique(np.sort(edges, axis=1), axis=0)
    mid = (kc[edges[:, 0]] + kc[edges[:, 1]]) // 2
    fm = lookup(mid)
    for e in range(2):
        rows.append(fm)
        cols.append(edges[:, e])
        vals.append(np.full(len(edges), 0.5))
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.mesh.n_nodes, coarse.mesh.n_nodes)).tocsr()
    return P


@dataclass
class Hierarchy:
    levels: dict                        # level -> StokesLevel
    P: dict = field(default_factory=dict)     # level -> P (fine l, coarse l-1), all nodes
    Pu: dict = field(default_factory=dict)    # level -> P restricted to free velocity nodes
    colours_u: dict = field(default_factory=dict)  # level -> [rows of colour c among free u]
    colours_p: dict = field(default_factory=dict)
    coarsest: int = 2
    finest: int = 2
    opt: Options = field(default_factory=Options)
    counts: dict | None = None   # optional: level -> {"A": n, "B": n, "C": n} operator applications

    def count(self, l: int, op: str, n: int = 1):
        if self.counts is not None:
            c = self.counts.setdefault(l, {"A": 0, "B": 0, "C": 0})
            c[op] += n


def build_hierarchy(macro, finest: int, coarsest: int = 2, nu: float = 1.0, delta: float = 1.0 / 12.0,
                    opt: Options | None = None, form: str = "laplace") -> Hierarchy:
    levels = {}
    for l in range(coarsest, finest + 1):
        mesh = refine(macro.vertices, macro.tets, macro.bc_flags, l, spacing=macro.spacing,
                      basis=getattr(macro, "basis", None))
        levels[l] = build_level(mesh, nu=nu, delta=delta, form=form)
    H = Hierarchy(levels=levels, coarsest=coarsest, finest=finest, opt=opt or Options())
    for l in range(coarsest, finest + 1):
        L = levels[l]
        col = colour_of(L)
        H.colours_u[l] = [np.where(col[L.free] == c)[0] for c in range(4)]
        H.colours_p[l] = [np.where(col == c)[0] for c in range(4)]
        if l > coarsest:
            P = prolongation(L, levels[l - 1])
            H.P[l] = P
            H.Pu[l] = P[L.free][:, levels[l - 1].free].tocsr()
    return H


# --- smoother ---------------------------------------------------------------

def _gs_sweep(Amat, diag, x, rhs, colour_rows, order, relax=1.0):
    """Colour-ordered Gauss-Seidel: for each colour, x_c += relax (rhs - A x)_c / diag_c."""
    for c in order:
        rows = colour_rows[c]
        if len(rows) == 0:
            continue
        r = rhs[rows] - Amat[rows] @ x
        x[rows] += relax * r / diag[rows]
    return x


def _block_gs_sweep(L: StokesLevel, u, rhs, colour_rows, order):
    """Colour-ordered block Gauss-Seidel on the coupled velocity block Kv (the
    D-form A2, free slip): for each colour, the velocity of its nodes (3
    components each) becomes u_c += D_c^-1 (rhs - Kv u)_c, D_c the nodes'
    3 x 3 diagonal blocks of Kv solved exactly.  Nodes of one colour are not
    coupled, so this equals a node-by-node block Gauss-Seidel in colour order."""
    for c in order:
        rows = colour_rows[c]
        if len(rows) == 0:
            continue
        r = (rhs - L.apply_A(u))[:, rows]                      # (3, nc)
        delta = np.linalg.solve(L.Kv_node[rows], r.T[:, :, None])[:, :, 0]
        u[:, rows] += delta.T
    return u


def uzawa_step(H: Hierarchy, l: int, u, p, f, g):
    """One inexact Uzawa smoothing step (Sec. 3.3) in place on (u, p).
    Velocity: SHGS, a forward and a backward colour Gauss-Seidel sweep on A
    with the right-hand side f - B^T p_k; in the D form (Sec. 2.1) on the
    coupled A2 with the 3 x 3 node blocks solved exactly (for the Laplace
    form these blocks are diagonal and the sweep is the component-wise one)."""
    L = H.levels[l]
    cu = H.colours_u[l]
    if L.coupled:
        H.count(l, "A", 2)
        H.count(l, "B", 2)
        H.count(l, "C", 1)
        rhs = L.proj(np.stack([f[d] - L.BT[d] @ p for d in range(3)]))
        _block_gs_sweep(L, u, rhs, cu, (0, 1, 2, 3))
        _block_gs_sweep(L, u, rhs, cu, (3, 2, 1, 0))
        up = L.proj(u)
        rhs_p = sum(L.B[d] @ up[d] for d in range(3)) - g
        _gs_sweep(L.C, L.C_diag, p, rhs_p, H.colours_p[l], (0, 1, 2, 3), relax=H.opt.omega)
        return u, p
    # operator applications in the counting of Sec. 4.2: the SHGS sweep pair
    # applies A twice, B^T p and B u are one B application each, the
    # pressure sweep applies C once
    H.count(l, "A", 2)
    H.count(l, "B", 2)
    H.count(l, "C", 1)
    for d in range(3):
        rhs = f[d] - L.BT[d] @ p
        _gs_sweep(L.A, L.A_diag, u[d], rhs, cu, (0, 1, 2, 3))
        _gs_sweep(L.A, L.A_diag, u[d], rhs, cu, (3, 2, 1, 0))
    rhs_p = sum(L.B[d] @ u[d] for d in range(3)) - g
    _gs_sweep(L.C, L.C_diag, p, rhs_p, H.colours_p[l], (0, 1, 2, 3), relax=H.opt.omega)
    return u, p


def smoothing_steps(H: Hierarchy, l: int, pre: bool = True, root: int | None = None, nu: int | None = None) -> int:
    """nu_l = nu + var_increment (root - l) on level l of a V_var(nu, nu) cycle
    rooted at level `root` (default: the finest level, nu: the options' nu_pre
    / nu_post); Sec. 3.5 for the solver cycle, Sec. 5 for the cycles of FMG."""
    base = (H.opt.nu_pre if pre else H.opt.nu_post) if nu is None else nu
    return base + H.opt.var_increment * ((H.finest if root is None else root) - l)


# --- coarse grid ------------------------------------------------------------

def coarse_solve(H: Hierarchy, f, g, history=None):
    """Block-preconditioned MINRES on the coarsest level, from zero (Sec. 3.7)."""
    L = H.levels[H.coarsest]
    o = H.opt
    nu = L.n_u

    def split(x):
        return x[:3 * nu].reshape(3, nu), x[3 * nu:]

    def apply_K(x):
        u, p = split(x)
        ru, rp = L.apply(u, p)
        return np.concatenate([ru.ravel(), rp])

    def apply_Pinv(x):
        u, p = split(x)
        if L.coupled:
            zu = krylov.cg(lambda v: L.Kv @ v, u.ravel(), o.coarse_cg_max, o.coarse_cg_rtol)
        else:
            zu = np.stack([krylov.cg(lambda v: L.A @ v, u[d], o.coarse_cg_max, o.coarse_cg_rtol) for d in range(3)])
        return np.concatenate([zu.ravel(), p / L.m])

    b = np.concatenate([f.ravel(), g])
    x = krylov.pminres(apply_K, b, apply_Pinv, o.coarse_minres_max, o.coarse_minres_rtol, history)
    return split(x)


# --- transfers ------------------------------------------------------------------

def restrict(H: Hierarchy, l: int, ru, rp):
    """Right-hand side of the coarse correction equation from the residual of
    level l: R = P^T for velocity and pressure (Sec. 3.5), the velocity
    projected on the admissible subspace at the coarse free-slip nodes
    (Sec. 6.1: the coarse correction is a constrained coarse velocity)."""
    Lc = H.levels[l - 1]
    return Lc.proj(np.stack([H.Pu[l].T @ ru[d] for d in range(3)])), H.P[l].T @ rp


def prolong(H: Hierarchy, l: int, uc, pc):
    """The coarse correction interpolated to level l by P, the velocity
    projected on the admissible subspace at the fine free-slip nodes (where
    the fine normals differ from the coarse ones, P uc is not tangential)."""
    L = H.levels[l]
    return L.proj(np.stack([H.Pu[l] @ uc[d] for d in range(3)])), H.P[l] @ pc


# --- cycle and solve ----------------------------------------------------------

def vcycle(H: Hierarchy, l: int, u, p, f, g, root: int | None = None, nu: int | None = None):
    """One V_var cycle on level l, in place on (u, p); smoothing counts as in
    smoothing_steps (root defaults to the finest level)."""
    if l == H.coarsest:
        # correction from the residual equation (inside a cycle u = p = 0 here)
        ru, rp = H.levels[l].residual(u, p, f, g)
        cu, cp = coarse_solve(H, ru, rp)
        u += cu
        p += cp
        return u, p
    L = H.levels[l]
    for _ in range(smoothing_steps(H, l, True, root, nu)):
        uzawa_step(H, l, u, p, f, g)
    ru, rp = L.residual(u, p, f, g)
    H.count(l, "A", 1)
    H.count(l, "B", 2)
    H.count(l, "C", 1)
    Lc = H.levels[l - 1]
    fc, gc = restrict(H, l, ru, rp)
    uc = np.zeros((3, Lc.n_u))
    pc = np.zeros(Lc.n_p)
    vcycle(H, l - 1, uc, pc, fc, gc, root, nu)
    du, dp = prolong(H, l, uc, pc)
    u += du
    p += dp
    for _ in range(smoothing_steps(H, l, False, root, nu)):
        uzawa_step(H, l, u, p, f, g)
    return u, p


@dataclass
class SolveResult:
    u: np.ndarray
    p: np.ndarray
    cycles: int
    history: list           # relative residual after each cycle (history[0] = 1)
    iterates: list          # (u, p) after each cycle, when requested


def solve(H: Hierarchy, f, g, u0=None, p0=None, tol: float = 1e-8, max_cycles: int = 50,
          keep_iterates: bool = False) -> SolveResult:
    L = H.levels[H.finest]
    u = np.zeros((3, L.n_u)) if u0 is None else np.array(u0, dtype=float, copy=True)
    p = np.zeros(L.n_p) if p0 is None else np.array(p0, dtype=float, copy=True)
    r0 = L.norm(*L.residual(u, p, f, g))
    hist = [1.0]
    its = []
    cycles = 0
    if r0 == 0.0:
        return SolveResult(u, p, 0, hist, its)
    for _ in range(max_cycles):
        vcycle(H, H.finest, u, p, f, g)
        p = L.project_pressure(p)
        cycles += 1
        rel = L.norm(*L.residual(u, p, f, g)) / r0
        hist.append(rel)
        if keep_iterates:
            its.append((u.copy(), p.copy()))
        if rel <= tol:
            break
    return SolveResult(u, p, cycles, hist, its)


# --- full multigrid (Sec. 5) ------------------------------------------------------

def fmg(H: Hierarchy, rhs: dict, dirichlet: dict, cycles: int = 1, nu: int = 2) -> SolveResult:
    """Full multigrid with `cycles` V_var(nu, nu) cycles per level (Sec. 5,
    Fig. "FMG": one cycle per level for "FMG V", two for "FMG 2V").

    rhs[l] = (f_l, g_l): the right-hand side rediscretised on level l;
    dirichlet[l]: (n_l, 3) nodal Dirichlet data of level l (None = 0).
    Starting from zero (Sec. 5), the coarsest level is solved by the coarse
    solver, and on every finer level l the iterate starts from the P1
    interpolant of the coarser level's whole velocity (Dirichlet values
    included) and pressure, followed by `cycles` V-cycles rooted at l with
    nu + var_increment (l - k) smoothing steps on level k; the pressure is
    projected to sum m p = 0 after each cycle on pure-Dirichlet meshes."""
    c = H.coarsest
    Lc = H.levels[c]
    u = np.zeros((3, Lc.n_u))
    p = np.zeros(Lc.n_p)
    f, g = rhs[c]
    vcycle(H, c, u, p, f, g)
    p = Lc.project_pressure(p)
    n_cycles = 0
    for l in range(c + 1, H.finest + 1):
        L, Lk = H.levels[l], H.levels[l - 1]
        full = Lk.scatter(u, dirichlet.get(l - 1))
        u = L.proj(np.stack([(H.P[l] @ full[:, d])[L.free] for d in range(3)]))
        p = H.P[l] @ p
        f, g = rhs[l]
        for _ in range(cycles):
            vcycle(H, l, u, p, f, g, root=l, nu=nu)
            p = L.project_pressure(p)
            n_cycles += 1
    Lf = H.levels[H.finest]
    f, g = rhs[H.finest]
    r0 = Lf.norm(f, g)
    rel = Lf.norm(*Lf.residual(u, p, f, g)) / r0 if r0 > 0 else 0.0
    return SolveResult(u, p, n_cycles, [1.0, rel], [])


def h_norm(L: StokesLevel, u, p) -> float:
    """Mesh-dependent norm of Sec. 5: (||u||_2^2 + h^2 ||p||_2^2)^(1/2) over the
    free velocity values and all pressure values of level L."""
    h = L.mesh.h
    return float(np.sqrt(np.sum(np.asarray(u) ** 2) + h * h * np.sum(np.asarray(p) ** 2)))
