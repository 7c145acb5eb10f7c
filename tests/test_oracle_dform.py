"""Pins of the oracle's D-operator formulation (Sec. 2.1: a_2(u, v) =
2 nu <D(u), D(v)>, D(u) = (grad u + grad u^T) / 2) and its smoother.

  * A2 is symmetric, and positive definite on the free velocity nodes.
  * Rigid motions u = c + w x x have D(u) = 0: A2 annihilates them on every
    row (A1 only on interior rows).
  * On functions vanishing on the boundary, int d_b u_a d_a v_b = int div u
    div v, so on the free x free block A2 = A1 (x) I + nu DivDiv with
    DivDiv[(i, a), (j, b)] = int d_a phi_i d_b phi_j, assembled here
    independently with the other index placement.
  * The exact states of the Laplace-form pins (hydrostatic, linear
    divergence-free Dirichlet flow) solve the D form too (D(G x) is constant).
  * The node-block colour Gauss-Seidel equals a node-by-node block loop, and
    its forward + backward pair is symmetric.
  * Cycle count at the paper's level 2: 9 (Tab. "itertime_D_ser"); the
    V-cycle converges to the direct solution.
  * Tab. "ratios_opcoutns": with the pinned operator counts of Sec. 4.2 and
    mu_d = 3.25, the D / Laplace ratio of total operator evaluations of UMG
    is 2.00 (the UMG counts are the same for both forms).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import direct, fem, multigrid as MG, stokes as S


def test_a2_symmetric_positive_definite():
    L = S.build_from_macro(W.unit_cube(), 2, form="D")
    assert abs(L.A2 - L.A2.T).max() <= 1e-15 * abs(L.A2).max()
    assert np.linalg.eigvalsh(L.A2.toarray()).min() > 0
    K = S.full_matrix(L)
    assert abs(K - K.T).max() == 0.0


def test_rigid_motions_in_kernel():
    """D(c + w x x) = 0 pointwise, so a_2(rigid, phi_i e_a) = 0 for every basis
    function, boundary ones included: A2 (all nodes) annihilates rigid
    motions on every row.  A1 does so only on interior rows."""
    L = S.build_from_macro(W.unit_cube(), 3, form="D", nu=1.3)
    x = L.mesh.xyz
    c, w = np.array([0.3, -1.1, 0.7]), np.array([0.9, 0.4, -1.6])
    u = c + np.cross(w, x)
    for a in range(3):
        row = sum(L.ops.A2[a][b] @ u[:, b] for b in range(3))
        assert np.abs(row).max() < 1e-13
    assert max(np.abs(L.ops.A @ u[:, a]).max() for a in range(3)) > 1e-3


def test_a2_equals_laplace_plus_divdiv_on_free_nodes():
    nu = 0.7
    L = S.build_from_macro(W.unit_cube(), 3, form="D", nu=nu)
    vol, grads = fem.element_geometry(L.mesh.xyz, L.mesh.tets)
    n = L.mesh.n_nodes
    zero = sp.csr_matrix((L.n_u, L.n_u))
    blocks = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            # test index m differentiated along a, trial index k along b
            loc = vol[:, None, None] * (grads[:, :, None, a] * grads[:, None, :, b])
            divdiv = fem._assemble(L.mesh.tets, loc, n)[L.free][:, L.free]
            blocks[a][b] = nu * divdiv + (L.A if a == b else zero)
    ref = sp.bmat(blocks, format="csr")
    assert abs(L.A2 - ref).max() <= 1e-12 * abs(L.A2).max()
    # the identity needs both functions to vanish on the boundary: with the
    # do-nothing outflow of the channel (free boundary nodes) it does not hold
    Lc = S.build_from_macro(W.obstacle_channel(), 1, form="D")
    assert abs(Lc.A2 - Lc.A2.T).max() == 0.0


@pytest.mark.parametrize("level", [2, 3])
def test_exact_states_solve_d_form(level):
    L = S.build_from_macro(W.unit_cube(), level, form="D")
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
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(u - u_lin[L.free].T).max() <= 1e-9 * np.abs(u_lin).max()


def _node_block_gs_brute(L, u, rhs, colours, order):
    A2 = L.A2.toarray()
    n = L.n_u
    y = u.copy().ravel()
    col = colours
    for c in order:
        nodes = np.where(col == c)[0]
        if order[0] > order[-1]:
            nodes = nodes[::-1]
        for i in nodes:
            idx = np.array([i, n + i, 2 * n + i])
            r = rhs.ravel()[idx] - A2[idx] @ y
            y[idx] += np.linalg.solve(A2[np.ix_(idx, idx)], r)
    return y.reshape(3, n)


def test_node_block_sweep_equals_sequential_and_shgs_symmetric():
    H = MG.build_hierarchy(W.unit_cube(), 2, form="D")
    L = H.levels[2]
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((3, L.n_u))
    rhs = rng.standard_normal((3, L.n_u))
    col = MG.colour_of(L)[L.free]
    for order in ((0, 1, 2, 3), (3, 2, 1, 0)):
        u = MG._block_gs_sweep(L, u0.copy(), rhs, H.colours_u[2], order)
        np.testing.assert_allclose(u, _node_block_gs_brute(L, u0, rhs, col, order), rtol=1e-12, atol=1e-12)
    # r -> u of the velocity half of an Uzawa step from zero is symmetric
    n = L.n_u
    Msm = np.zeros((3 * n, 3 * n))
    for j in range(3 * n):
        u = np.zeros((3, n))
        f = np.zeros(3 * n)
        f[j] = 1.0
        MG.uzawa_step(H, 2, u, np.zeros(L.n_p), f.reshape(3, n), np.zeros(L.n_p))
        Msm[:, j] = u.ravel()
    assert np.abs(Msm - Msm.T).max() <= 1e-13 * np.abs(Msm).max()


def test_d_form_cycle_count_and_direct_solution():
    H = MG.build_hierarchy(W.unit_cube(), 4, form="D")
    L = H.levels[4]
    x = L.mesh.xyz
    f, g = L.rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    res = MG.solve(H, f, g, tol=1e-8, max_cycles=30)
    assert abs(res.cycles - 9) <= 1   # Tab. "itertime_D_ser", UMG at L = 2: 9
    H3 = MG.build_hierarchy(W.unit_cube(), 3, form="D")
    L3 = H3.levels[3]
    f3, g3 = L3.rhs(W.manufactured_forcing(L3.mesh.xyz), W.manufactured_velocity(L3.mesh.xyz))
    r3 = MG.solve(H3, f3, g3, tol=1e-13, max_cycles=60)
    ud, pd = direct.solve_direct(L3, f3, g3)
    assert np.abs(r3.u - ud).max() <= 1e-9 * np.abs(ud).max()
    assert np.abs(r3.p - pd).max() <= 1e-8 * np.abs(pd).max()


def test_operator_count_ratio_matches_paper(golden):
    oc = golden["operator_counts_L6"]
    mu_d = 3.25
    lap = 3 * oc["A"] + 3 * oc["B"] + oc["C"]
    dform = 3 * mu_d * oc["A"] + 3 * oc["B"] + oc["C"]
    assert dform / lap == pytest.approx(2.00, abs=0.005)


@pytest.mark.parametrize("macro_name,level", [("cube", 2), ("channel", 1)])
@pytest.mark.parametrize("form", ["laplace", "D"])
def test_dirichlet_lift_from_the_bilinear_form(form, macro_name, level):
    """The lift of the right-hand side (Sec. 2.1) is f_{i,a} = -a(w, phi_i e_a)
    with w the interpolant of the Dirichlet data.  Computed here element by
    element from the gradient of w, not from the assembled blocks:
    a_1(w, phi_i e_a) = nu sum_T |T| (grad w grad phi_i)_a and
    a_2(w, phi_i e_a) = 2 nu sum_T |T| (D(w) grad phi_i)_a, D(w) the
    symmetric part of grad w (D(phi_i e_a) : D(w) = (D(w) grad phi_i)_a).
    A_2 and its block transpose differ by a null Lagrangian, int (grad v :
    grad w^T - div v div w), which vanishes for test functions that vanish on
    the boundary: only rows of free boundary nodes (the channel's outflow
    face) tell them apart, so the channel is checked beside the cube."""
    macro = W.unit_cube() if macro_name == "cube" else W.obstacle_channel()
    L = S.build_from_macro(macro, level, form=form)
    x = L.mesh.xyz
    ud = np.stack([np.sin(3 * x[:, 1]) + x[:, 0] ** 2, x[:, 2] * x[:, 0], np.cos(2 * x[:, 0] + x[:, 1])], axis=1)
    w = np.zeros_like(ud)
    w[L.dir] = ud[L.dir]
    fu, _ = L.rhs(None, ud)
    vol, grads = fem.element_geometry(x, L.mesh.tets)
    gw = np.einsum("tmi,tmj->tij", w[L.mesh.tets], grads)   # (grad w)_ij = d_j w_i per element
    Mt = 0.5 * (gw + np.transpose(gw, (0, 2, 1))) if form == "D" else gw
    fac = 2.0 if form == "D" else 1.0
    contrib = -fac * vol[:, None, None] * np.einsum("tij,tmj->tmi", Mt, grads)   # (nT, 4, 3)
    ref = np.zeros_like(ud)
    for m in range(4):
        np.add.at(ref, L.mesh.tets[:, m], contrib[:, m])
    np.testing.assert_allclose(fu.T, ref[L.free], rtol=0, atol=1e-13 * np.abs(ref[L.free]).max())
