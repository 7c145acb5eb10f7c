"""Pins of the oracle's element integrals and assembly (Sec. 2.1).

Checked against facts derived independently of the assembly code:
  * closed-form interior rows on the Kuhn lattice (worked out by hand from
    the barycentric gradients of a Kuhn tetrahedron): A is the 7-point
    Laplacian nu*h*(6, -1 x 6); C is delta*h_T^2*h*(same); B_d is the
    antisymmetric 14-point row with weights h^2/4 and h^2/12; M has the
    15-point row h^3 (2/5, 1/20 on axis and body-diagonal offsets, 1/30 on
    face diagonals);
  * consistency: A and C annihilate linear functions on interior rows,
    B_d x_d = -m on every row (int phi_i div(x_d e_d) = int phi_i), B^T 1 = 0
    on interior velocity rows, C 1 = 0, 1^T M 1 = |Omega|, M 1 = m,
    G f = 0 on interior rows for a constant f;
  * symmetry of K and positive definiteness of A on free nodes;
  * Galerkin identities of the nested P1 spaces: A_c = P^T A_f P,
    B_c = P^T B_f P, M_c = P^T M_f P, and C_c = 4 P^T C_f P (h_T doubles);
    P reproduces linear functions.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, mesh as M, multigrid as MG, stokes as S


@pytest.fixture(scope="module")
def cube3():
    cube = W.unit_cube()
    m = M.refine(cube.vertices, cube.tets, cube.bc_flags, 3)
    return m, fem.assemble(m, nu=1.7, delta=1.0 / 12.0)


def _row(Mx, m, node):
    row = Mx.getrow(node)
    tiny = 1e-13 * np.abs(row.data).max()   # drop cancellation roundoff
    return {tuple(m.ijk[j] - m.ijk[node]): v for j, v in zip(row.indices, row.data) if abs(v) > tiny}


def _interior(m):
    return np.where(np.all((m.ijk > 0) & (m.ijk < m.N), axis=1))[0]


def test_closed_form_rows(cube3):
    m, ops = cube3
    h, nu = m.h, 1.7
    hT2 = (h ** 3 / 6.0) ** (2.0 / 3.0)
    axis = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    face = [(1, 1, 0), (0, 1, 1), (1, 0, 1)]
    body = (1, 1, 1)
    for node in _interior(m)[::37]:
        a = _row(ops.A, m, node)
        expect = {(0, 0, 0): 6 * nu * h}
        for o in axis:
            expect[o] = expect[tuple(-x for x in o)] = -nu * h
        assert a.keys() == expect.keys()
        for k in a:
            assert a[k] == pytest.approx(expect[k], rel=1e-12)
        c = _row(ops.C, m, node)
        for k in c:
            assert c[k] == pytest.approx(expect[k] / nu * hT2 / 12.0, rel=1e-12)
        mm = _row(ops.M, m, node)
        h3 = h ** 3
        assert mm[(0, 0, 0)] == pytest.approx(0.4 * h3)
        for o in axis + [body]:
            assert mm[o] == pytest.approx(h3 / 20) and mm[tuple(-x for x in o)] == pytest.approx(h3 / 20)
        for o in face:
            assert mm[o] == pytest.approx(h3 / 30) and mm[tuple(-x for x in o)] == pytest.approx(h3 / 30)
        for d in range(3):
            b = _row(ops.B[d], m, node)
            assert len(b) == 14 and (0, 0, 0) not in b
            for o, v in b.items():
                assert b[tuple(-x for x in o)] == pytest.approx(-v, rel=1e-12)  # antisymmetric
            # weights on the positive half: -1/4 on e_d, +1/12 on the other axes,
            # -1/12 on face diagonals containing e_d, +1/12 on the one that does not,
            # -1/12 on the body diagonal
            for o in axis:
                want = -0.25 if o[d] else 1.0 / 12.0
                assert b[o] == pytest.approx(want * h * h, rel=1e-12)
            for o in face:
                want = -1.0 / 12.0 if o[d] else 1.0 / 12.0
                assert b[o] == pytest.approx(want * h * h, rel=1e-12)
            assert b[body] == pytest.approx(-h * h / 12.0, rel=1e-12)


def test_consistency_invariants(cube3):
    m, ops = cube3
    x = m.xyz
    inner = _interior(m)
    lin = 0.3 + 1.1 * x[:, 0] - 0.7 * x[:, 1] + 2.0 * x[:, 2]
    assert np.abs((ops.A @ lin)[inner]).max() < 1e-13
    assert np.abs((ops.C @ lin)[inner]).max() < 1e-15
    for d in range(3):
        np.testing.assert_allclose(ops.B[d] @ x[:, d], -ops.m, rtol=1e-12, atol=1e-16)
        assert np.abs((ops.B[d].T @ np.ones(m.n_nodes))[inner]).max() < 1e-15
        assert np.abs((ops.G[d] @ np.ones(m.n_nodes))[inner]).max() < 1e-17
    assert np.abs(ops.C @ np.ones(m.n_nodes)).max() < 1e-16
    assert np.ones(m.n_nodes) @ ops.M @ np.ones(m.n_nodes) == pytest.approx(1.0, rel=1e-13)
    np.testing.assert_allclose(ops.M @ np.ones(m.n_nodes), ops.m, rtol=1e-13)
    # int x over the unit cube
    assert np.ones(m.n_nodes) @ ops.M @ x[:, 0] == pytest.approx(0.5, rel=1e-13)


def test_symmetry_and_spd():
    cube = W.unit_cube()
    L = S.build_from_macro(cube, 2)
    K = S.full_matrix(L)
    assert abs(K - K.T).max() == 0.0
    ev = np.linalg.eigvalsh(L.A.toarray())
    assert ev.min() > 0
    # K has exactly one zero eigenvalue in the pure-Dirichlet case: (0, 1)
    evK = np.linalg.eigvalsh(K.toarray())
    assert np.sum(np.abs(evK) < 1e-12 * np.abs(evK).max()) == 1


@pytest.mark.parametrize("macro_name", ["cube", "channel"])
def test_galerkin_identities(macro_name):
    macro = W.unit_cube() if macro_name == "cube" else W.obstacle_channel()
    lf, lc = (3, 2) if macro_name == "cube" else (1, 0)
    Lf = S.build_from_macro(macro, lf, nu=1.3)
    Lc = S.build_from_macro(macro, lc, nu=1.3)
    P = MG.prolongation(Lf, Lc)
    def close(X, Y):
        D = (X - Y).tocsr()
        return abs(D).max() <= 1e-12 * abs(Y).max()
    assert close(P.T @ Lf.ops.A @ P, Lc.ops.A)
    assert close(P.T @ Lf.ops.M @ P, Lc.ops.M)
    assert close(4.0 * (P.T @ Lf.ops.C @ P), Lc.ops.C)
    for d in range(3):
        assert close(P.T @ Lf.ops.B[d] @ P, Lc.ops.B[d])
        assert close(4.0 * (P.T @ Lf.ops.G[d] @ P), Lc.ops.G[d])
    # P reproduces linear functions and has unit row sums
    lin_c = 1.0 + Lc.mesh.xyz @ np.array([0.5, -2.0, 3.0])
    lin_f = 1.0 + Lf.mesh.xyz @ np.array([0.5, -2.0, 3.0])
    np.testing.assert_allclose(P @ lin_c, lin_f, rtol=0, atol=1e-12)
    assert set(np.unique(P.data)) <= {0.5, 1.0}


def test_outflow_weights():
    """int over the outflow face of phi_i n sums to the face area times n."""
    ch = W.obstacle_channel()
    m = M.refine(ch.vertices, ch.tets, ch.bc_flags, 1)
    ops = fem.assemble(m)
    np.testing.assert_allclose(ops.w_out.sum(axis=0), [16.0, 0.0, 0.0], atol=1e-12)
    assert np.all(ops.w_out[~M.node_on_outflow_face(m)] == 0.0)
