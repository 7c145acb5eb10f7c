"""Pins of the oracle by problems whose discrete solution is known exactly,
and by the symmetry of the SHGS velocity smoother.

Exact discrete solutions (Sec. 2.1 forms: a_1, b(v, q) = -<div v, q>, the
PSPG terms c_l and g_l = -sum_T delta h_T^2 <f, grad q>_T):

  * Hydrostatic state.  For a body force f = grad(phi) with phi linear and
    homogeneous Dirichlet velocity, (u_h, p_h) = (0, I_h phi) solves the
    discrete system exactly: b(v, phi) = <grad phi, v> for every v vanishing
    on the Dirichlet boundary (and on an outflow face where phi = 0), and the
    second equation reads -c_l(phi, q) = g_l(q), which holds with the sign of
    g_l as printed because f = grad(phi) element by element.  A wrong sign of
    g_l, of B or of B^T breaks it.  On the cube the pressure is defined up to
    a constant and fixed by sum_i m_i p_i = 0.
  * Linear divergence-free flow.  With f = 0 and Dirichlet data u_D = G x,
    trace G = 0, on the cube, (I_h u_D, 0) solves the system exactly:
    a_1(G x, v) = 0 for v vanishing on the boundary (constant gradient) and
    b(G x, q) = 0 (div = 0 pointwise).  It pins the Dirichlet lift
    f <- f - A_{I,D} u_D, g <- g - B_{.,D} u_D, its signs included.

SHGS (Sec. 3.4-3.5): one forward Gauss-Seidel sweep followed by one backward
sweep from zero on the same right-hand side is the symmetric Gauss-Seidel
preconditioner (D + U)^-1 D (D + L)^-1, a symmetric matrix when A is.  With
colours visited 0,1,2,3 forward and 3,2,1,0 backward (block Gauss-Seidel
with diagonal colour blocks) the map r -> u of the velocity half of an
Uzawa step from (u, p) = 0 must be symmetric; sweeping forward twice is not.

Tolerances: the residual of the exact state is zero to 1e-13 relative to the
right-hand side (no solve involved: the sharp pin); the direct solution agrees
with it to 1e-9 and the multigrid solution (relative residual 1e-13) to 1e-8
(rounding and residual grow into the pressure with the condition number of
K); a wrong sign anywhere gives O(1) differences.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct, multigrid as MG, stokes as S


def _phi(x, c0, grad):
    return c0 + x @ np.asarray(grad, float)


def _grad_field(x, grad):
    return np.broadcast_to(np.asarray(grad, float), x.shape).copy()


@pytest.mark.parametrize("level", [2, 3])
def test_hydrostatic_cube(level):
    L = S.build_from_macro(W.unit_cube(), level)
    x = L.mesh.xyz
    grad = (1.7, -0.6, 2.3)
    f, g = L.rhs(_grad_field(x, grad), None)
    u, p = direct.solve_direct(L, f, g)
    phi = _phi(x, 0.4, grad)
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    assert np.abs(u).max() <= 1e-9 * np.abs(p_ref).max()
    assert np.abs(p - p_ref).max() <= 1e-9 * np.abs(p_ref).max()
    # and the residual of the exact state is zero (no direct solve involved)
    ru, rp = L.residual(np.zeros_like(u), p_ref, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale


def test_hydrostatic_channel():
    """Channel with obstacles and a do-nothing outflow on x = 16: phi = a (x - 16)
    vanishes on the outflow face, so the natural boundary term is zero and
    (0, phi) is the exact solution; no mean projection (K is regular)."""
    ch = W.obstacle_channel()
    L = S.build_from_macro(ch, 1)
    assert not L.pure_dirichlet
    x = L.mesh.xyz
    a = 0.75
    f, g = L.rhs(_grad_field(x, (a, 0.0, 0.0)), None)
    phi = a * (x[:, 0] - 16.0)
    ru, rp = L.residual(np.zeros((3, L.n_u)), phi, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(u).max() <= 1e-9 * np.abs(phi).max()
    assert np.abs(p - phi).max() <= 1e-9 * np.abs(phi).max()


@pytest.mark.parametrize("level", [2, 3])
def test_linear_flow_and_hydrostatic_superposed(level):
    L = S.build_from_macro(W.unit_cube(), level)
    x = L.mesh.xyz
    G = np.array([[0.5, 1.2, -0.3], [0.7, -1.5, 0.4], [-0.9, 0.2, 1.0]])  # trace 0
    assert abs(np.trace(G)) < 1e-15
    u_lin = x @ G.T + np.array([0.1, -0.2, 0.3])
    grad = (-1.1, 0.8, 0.5)
    f, g = L.rhs(_grad_field(x, grad), u_lin)
    phi = _phi(x, 0.0, grad)
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    u_ref = u_lin[L.free].T
    ru, rp = L.residual(u_ref, p_ref, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert np.abs(p - p_ref).max() <= 1e-9 * np.abs(p_ref).max()
    # the multigrid solve reaches the same exact state
    H = MG.build_hierarchy(W.unit_cube(), level)
    Lm = H.levels[level]
    fm, gm = Lm.rhs(_grad_field(Lm.mesh.xyz, grad), u_lin)
    res = MG.solve(H, fm, gm, tol=1e-13, max_cycles=60)
    assert np.abs(res.u - u_ref).max() <= 1e-8 * np.abs(u_ref).max()
    assert np.abs(res.p - p_ref).max() <= 1e-8 * np.abs(p_ref).max()


def _velocity_smoother_matrix(H, l):
    """Column by column: r -> u after one Uzawa step from (u, p) = (0, 0) with
    f = r e_0-component, g = 0 (the pressure half runs after the velocity half
    and does not change u)."""
    L = H.levels[l]
    n = L.n_u
    Msm = np.zeros((n, n))
    for j in range(n):
        u = np.zeros((3, n))
        p = np.zeros(L.n_p)
        f = np.zeros((3, n))
        f[0, j] = 1.0
        MG.uzawa_step(H, l, u, p, f, np.zeros(L.n_p))
        Msm[:, j] = u[0]
        assert np.all(u[1:] == 0.0)
    return Msm


@pytest.mark.parametrize("macro_name,level,coarsest", [("cube", 2, 2), ("channel", 1, 1)])
def test_shgs_is_symmetric(macro_name, level, coarsest):
    macro = W.unit_cube() if macro_name == "cube" else W.obstacle_channel()
    H = MG.build_hierarchy(macro, level, coarsest=coarsest)
    Msm = _velocity_smoother_matrix(H, level)
    assert np.abs(Msm - Msm.T).max() <= 1e-13 * np.abs(Msm).max()
    # it is the symmetric Gauss-Seidel preconditioner of A in colour order
    L = H.levels[level]
    perm = np.concatenate(H.colours_u[level])
    Ap = L.A.toarray()[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    Lo = np.tril(Ap, -1)
    Up = np.triu(Ap, 1)
    sgs = np.linalg.solve(D + Up, D @ np.linalg.inv(D + Lo))
    ref = np.zeros_like(sgs)
    ref[np.ix_(perm, perm)] = sgs
    np.testing.assert_allclose(Msm, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_backward_colour_sweep_equals_sequential_gs():
    """The backward sweep (colours 3, 2, 1, 0) equals a node-by-node loop over
    the colours in descending order."""
    H = MG.build_hierarchy(W.unit_cube(), 2)
    L = H.levels[2]
    rng = np.random.default_rng(6)
    x0 = rng.standard_normal(L.n_u)
    rhs = rng.standard_normal(L.n_u)
    x = MG._gs_sweep(L.A, L.A_diag, x0.copy(), rhs, H.colours_u[2], (3, 2, 1, 0))
    Ad = L.A.toarray()
    y = x0.copy()
    col = MG.colour_of(L)[L.free]
    for c in (3, 2, 1, 0):
        for i in np.where(col == c)[0][::-1]:
            y[i] += (rhs[i] - Ad[i] @ y) / Ad[i, i]
    np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("form", ["laplace", "D"])
def test_exact_states_on_sheared_cube(form):
    """The hydrostatic and linear-flow states are exact on any mesh, here the
    sheared cube (tetrahedra not aligned with the axes), in both forms."""
    L = S.build_from_macro(W.sheared_cube(), 2, form=form)
    x = L.mesh.xyz
    G = np.array([[0.5, 1.2, -0.3], [0.7, -1.5, 0.4], [-0.9, 0.2, 1.0]])
    u_lin = x @ G.T + np.array([0.1, -0.2, 0.3])
    grad = np.array([-1.1, 0.8, 0.5])
    f, g = L.rhs(np.broadcast_to(grad, x.shape).copy(), u_lin)
    phi = x @ grad
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    ru, rp = L.residual(u_lin[L.free].T, p_ref, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale
    H = MG.build_hierarchy(W.sheared_cube(), 2)
    assert MG.colouring_is_valid(H.levels[2])
