"""Oracle: outflow functional and its gradient w.r.t. the body force (test infrastructure).

The functional is a weighted volume flux through the do-nothing boundary,
    J = sum_i psi_i w_i . u_i,   w_i = int_{Gamma_out} phi_i n dS,
with nodal weights psi (psi = 1 is the plain flux int_{Gamma_out} u_h . n).
The plain flux does not depend on f at all: q = 1 is a pressure test
function, c_l(1, p) = 0 and g_l(1) = 0, so b(u_h, 1) = 0 and the flux out
equals the flux of the Dirichlet data in; its gradient is zero.
for the discrete solution of the system of Sec. 3 with a nodal body force f
(an input; Sec. 6 uses f = 0, the gradient study perturbs it).  The map from
f to the right-hand side is linear,
    R f = ( (M f_d)[free] for d = 0,1,2 ;  sum_d G_d f_d ),
so J is affine in f and, K being symmetric (Sec. 3),
    dJ/df = R^T K^{-1} j,   j = (psi w restricted to free velocity nodes, 0).
Only problems with an outflow boundary are handled here (K is then
non-singular).
"""
from __future__ import annotations

import numpy as np

from .direct import solve_direct
from .stokes import StokesLevel


def weights(L: StokesLevel, psi=None) -> np.ndarray:
    """Nodal weights W_i = psi_i w_i of the functional, (n, 3)."""
    w = L.ops.w_out
    return w if psi is None else w * np.asarray(psi)[:, None]


def functional(L: StokesLevel, u_free: np.ndarray, u_dirichlet=None, psi=None) -> float:
    u = L.scatter(u_free, u_dirichlet)
    return float(np.sum(weights(L, psi) * u))


def adjoint_rhs(L: StokesLevel, psi=None):
    W = weights(L, psi)
    ju = np.stack([W[L.free, d] for d in range(3)])
    return ju, np.zeros(L.n_p)


def rhs_transpose(L: StokesLevel, lam_u: np.ndarray, lam_p: np.ndarray) -> np.ndarray:
    """R^T (lam_u, lam_p) as a nodal field (n, 3)."""
    n = L.mesh.n_nodes
    out = np.zeros((n, 3))
    for d in range(3):
        full = np.zeros(n)
        full[L.free] = lam_u[d]
        out[:, d] = L.ops.M.T @ full + L.ops.G[d].T @ lam_p
    return out


def gradient_direct(L: StokesLevel, psi=None) -> np.ndarray:
    """dJ/df by one direct adjoint solve."""
    if L.pure_dirichlet:
        raise NotImplementedError("adjoint oracle needs an outflow boundary")
    lu, lp = solve_direct(L, *adjoint_rhs(L, psi))
    return rhs_transpose(L, lu, lp)


def functional_direct(L: StokesLevel, f_nodal, u_dirichlet, psi=None) -> float:
    f, g = L.rhs(f_nodal, u_dirichlet)
    u, _ = solve_direct(L, f, g)
    return functional(L, u, u_dirichlet, psi)
