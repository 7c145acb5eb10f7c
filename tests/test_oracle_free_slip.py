"""Pins of the oracle's free-slip boundary condition (Sec. 6.1).

The paper imposes u . n = 0 and a vanishing tangential stress point-wise at
the nodes of free-slip faces, with the mass-conservative normal
n_i = <grad phi_i, 1> / |<grad phi_i, 1>|.  The oracle solves the system
with the velocity block Pi A Pi + (I - Pi) and the coupling blocks Pi B^T,
B Pi (Pi = I - n n^T at slip nodes).  What fixes it independently:

  * the normals: <grad phi_i, 1> is the surface integral of phi_i n over the
    boundary (divergence theorem); assembled here from the fine boundary
    triangles (area / 3 per vertex times the outward unit normal), without
    B.  On a flat face it is the face normal;
  * mass conservation: sum_j (B u)_j = -sum_i <grad phi_i, 1> . u_i, and a
    slip node's term vanishes exactly when its admissible velocities are
    orthogonal to <grad phi_i, 1> (the tangent plane of the mass-conservative
    normal; along an obstacle edge, the edge direction), so the flux out of
    the channel equals the interpolated inflow with free-slip obstacles; with
    one face's normal at the edge nodes it does not;
  * exact states on the cube with free-slip faces x = 0 and x = 1: a linear
    divergence-free flow tangential to them with no x-dependence of its
    tangential part satisfies both the Laplace and the D-form natural
    condition, and a hydrostatic pressure adds f = grad(phi); both solve the
    discrete system exactly;
  * symmetry of the constrained K and of the SHGS velocity smoother, and the
    node update of a slip node equal to the tangential part of the
    unconstrained update (the form the GPU kernels take);
  * multigrid converges to the direct solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, direct, mesh as M, multigrid as MG, stokes as S

from test_oracle_exact_solutions import _velocity_smoother_matrix


def _surface_normals(L):
    """sum over boundary triangles of (area / 3) n at each vertex: the
    boundary integral of phi_i n, by the divergence theorem equal to
    <grad phi_i, 1>."""
    mesh = L.mesh
    faces = {}
    for t, tet in enumerate(mesh.tets):
        for f in range(4):
            key = tuple(sorted(int(v) for m, v in enumerate(tet) if m != f))
            faces.setdefault(key, []).append((t, f))
    acc = np.zeros((mesh.n_nodes, 3))
    for key, owners in faces.items():
        if len(owners) != 1:
            continue
        t, f = owners[0]
        a, b, c = (mesh.xyz[v] for v in key)
        nrm = np.cross(b - a, c - a)
        opp = mesh.xyz[mesh.tets[t][f]]
        if np.dot(nrm, opp - a) > 0:
            nrm = -nrm
        # |cross| = 2 area; area / 3 per vertex
        for v in key:
            acc[v] += nrm / 6.0
    return acc


@pytest.mark.parametrize("name,level", [("cube", 2), ("channel", 1), ("channel", 2)])
def test_normals_are_surface_integrals(name, level):
    macro = W.slip_cube() if name == "cube" else W.slip_channel()
    L = S.build_from_macro(macro, level)
    assert len(L.slip) > 0
    surf = _surface_normals(L)
    acc = surf[L.free[L.slip]]
    ref = acc / np.linalg.norm(acc, axis=1)[:, None]
    assert np.abs(L.normals - ref).max() <= 1e-13
    # nodes of slip faces whose integral vanishes (obstacles touching along an
    # edge) have no normal: they are Dirichlet nodes
    fresh = M.refine(macro.vertices, macro.tets, macro.bc_flags, level)
    pinch = fresh.on_slip & (np.linalg.norm(surf, axis=1) <= 1e-12)
    assert not np.isin(np.where(pinch)[0], L.free).any()
    if name == "channel":
        assert pinch.sum() == 2 ** level - 1  # the interior nodes of the one contact edge of seed 0
    if name == "cube":
        # every slip node lies inside a face x = 0 or x = 1: n = -e_x or +e_x
        x = L.mesh.xyz[L.free[L.slip]]
        assert set(np.round(x[:, 0], 12)) == {0.0, 1.0}
        exp = np.zeros_like(ref)
        exp[:, 0] = np.where(x[:, 0] == 0.0, -1.0, 1.0)
        assert np.abs(L.normals - exp).max() <= 1e-15


def test_slip_nodes_exclude_dirichlet_rim():
    L = S.build_from_macro(W.slip_cube(), 3)
    x = L.mesh.xyz[L.free[L.slip]]
    inner = (x[:, 1] > 0) & (x[:, 1] < 1) & (x[:, 2] > 0) & (x[:, 2] < 1)
    assert inner.all() and len(x) == 2 * 7 * 7


def test_constrained_system_is_symmetric_with_normal_identity():
    L = S.build_from_macro(W.slip_channel(), 1)
    K = S.full_matrix(L)
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    # the velocity block acts as the identity on each slip node's normal direction
    n = L.n_u
    for q in (0, len(L.slip) // 2, len(L.slip) - 1):
        i = L.slip[q]
        v = np.zeros(3 * n)
        v[np.arange(3) * n + i] = L.normals[q]
        w = L.Kv @ v
        exp = np.zeros(3 * n)
        exp[np.arange(3) * n + i] = L.normals[q]
        assert np.abs(w - exp).max() <= 1e-14
    # Pi_i B^T 1 = 0 at slip nodes: the pressure constant stays in the kernel
    bt1 = L.proj(np.stack([L.BT[d] @ np.ones(L.n_p) for d in range(3)]))
    assert np.abs(bt1[:, L.slip]).max() <= 1e-15 * np.abs(bt1).max()


def _channel_flux_balance(L, u, uD):
    flux_out = adjoint.functional(L, u, uD)
    full = np.zeros(L.mesh.n_nodes)
    full[L.dir] = uD[L.dir, 0]
    flux_in = float(np.sum(L.ops.B[0] @ full))
    return flux_out, flux_in


def test_mass_conservation_with_free_slip_obstacles():
    ch = W.slip_channel()
    L = S.build_from_macro(ch, 1)
    uD = W.channel_inflow(L.mesh.xyz)
    f, g = L.rhs(None, uD)
    u, p = direct.solve_direct(L, f, g)
    u_full = L.scatter(u, uD)
    # the slip velocities are tangential
    assert np.abs(np.sum(u[:, L.slip].T * L.normals, axis=1)).max() <= 1e-12 * np.abs(u).max()
    out, inn = _channel_flux_balance(L, u, uD)
    assert out == pytest.approx(inn, rel=1e-11)
    total = sum(float(np.sum(L.ops.B[d] @ u_full[:, d])) for d in range(3))
    assert abs(total) <= 1e-11 * abs(out)
    # the flow differs from the no-slip solution (the obstacles let it slide)
    L0 = S.build_from_macro(W.obstacle_channel(), 1)
    f0, g0 = L0.rhs(None, uD)
    u0, _ = direct.solve_direct(L0, f0, g0)
    assert np.abs(L0.scatter(u0, uD) - u_full).max() > 1e-2

    # edge nodes are constrained along the edge: orthogonal to both faces'
    # normals and to the mass-conservative normal
    assert L.slip_edge.any() and not L.slip_edge.all()
    Pe = L.slip_P[L.slip_edge]
    assert np.abs(np.einsum("nab,nb->na", Pe, L.normals[L.slip_edge])).max() <= 1e-13
    assert np.allclose(np.einsum("naa->n", Pe), 1.0)
    # the same system with one face's normal at the edge nodes loses the flux balance
    Lg = S.build_from_macro(ch, 1)
    ax = np.argmax(np.abs(Lg.normals), axis=1)
    one = np.zeros_like(Lg.normals)
    one[np.arange(len(ax)), ax] = np.sign(Lg.normals[np.arange(len(ax)), ax])
    P1 = np.eye(3)[None] - one[:, :, None] * one[:, None, :]
    Lg.slip_P = np.where(Lg.slip_edge[:, None, None], P1, Lg.slip_P)
    S.couple(Lg)
    ug, _ = direct.solve_direct(Lg, *Lg.rhs(None, uD))
    out_g, inn_g = _channel_flux_balance(Lg, ug, uD)
    assert abs(out_g - inn_g) > 1e-6 * abs(inn_g)


def _face_mean_normals(L):
    """Mean of the unit normals of the boundary faces incident to each slip
    node (area-independent): a plausible but not mass-conservative choice."""
    mesh = L.mesh
    faces = {}
    for t, tet in enumerate(mesh.tets):
        for f in range(4):
            key = tuple(sorted(int(v) for m, v in enumerate(tet) if m != f))
            faces.setdefault(key, []).append((t, f))
    dirs = {}
    for key, owners in faces.items():
        if len(owners) != 1:
            continue
        t, f = owners[0]
        a, b, c = (mesh.xyz[v] for v in key)
        nrm = np.cross(b - a, c - a)
        if np.dot(nrm, mesh.xyz[mesh.tets[t][f]] - a) > 0:
            nrm = -nrm
        nrm = tuple(np.round(nrm / np.linalg.norm(nrm), 12))
        for v in key:
            dirs.setdefault(v, set()).add(nrm)
    out = []
    for i in L.free[L.slip]:
        s = np.sum(np.array(sorted(dirs[i])), axis=0)
        nrm = np.linalg.norm(s)
        out.append(s / nrm if nrm > 1e-12 else np.zeros(3))
    return np.array(out)


def _slip_cube_state(x):
    """u = (0, a y + b z + c, d y - a z + e): no x-component, tangential parts
    independent of x, divergence free; p = phi linear."""
    a, b, c, d, e = 0.7, -1.2, 0.3, 0.9, -0.4
    u = np.stack([np.zeros(len(x)), a * x[:, 1] + b * x[:, 2] + c, d * x[:, 1] - a * x[:, 2] + e], axis=1)
    grad = np.array([1.3, -0.5, 0.8])
    return u, grad


@pytest.mark.parametrize("form", ["laplace", "D"])
@pytest.mark.parametrize("level", [2, 3])
def test_exact_state_on_slip_cube(form, level):
    L = S.build_from_macro(W.slip_cube(), level, form=form)
    x = L.mesh.xyz
    u_ex, grad = _slip_cube_state(x)
    f, g = L.rhs(np.broadcast_to(grad, x.shape).copy(), u_ex)
    phi = x @ grad
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    u_ref = u_ex[L.free].T
    ru, rp = L.residual(u_ref, p_ref, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert np.abs(p - p_ref).max() <= 1e-9 * np.abs(p_ref).max()
    # a flow with an x-dependent tangential part violates the natural
    # condition and is not a discrete solution
    u_bad = u_ex.copy()
    u_bad[:, 1] += 0.5 * x[:, 0] * (1.0 - x[:, 0])
    fb, gb = L.rhs(np.broadcast_to(grad, x.shape).copy(), u_bad)
    rub, _ = L.residual(u_bad[L.free].T, p_ref, fb, gb)
    assert np.abs(rub).max() > 1e-3 * scale


@pytest.mark.parametrize("form", ["laplace", "D"])
def test_slip_node_update_is_tangential_part_of_free_update(form):
    """Block Gauss-Seidel on Pi A Pi + (I - Pi) at a slip node, from an
    admissible iterate, equals: Laplace form, the unconstrained
    component-wise update projected on the node's admissible subspace (the
    tangent plane, or the edge direction at obstacle edges); D form,
    Z (rhs - off-diagonal row) with Z = T (T^T A_ii T)^-1 T^T, T an
    orthonormal basis of that subspace."""
    L = S.build_from_macro(W.slip_channel(), 1, form=form)
    rng = np.random.default_rng(3)
    u = L.proj(rng.standard_normal((3, L.n_u)))
    rhs = rng.standard_normal((3, L.n_u))
    edges = np.where(L.slip_edge)[0]
    planes = np.where(~L.slip_edge)[0]
    for q in (planes[0], planes[-1], edges[0], edges[-1]):
        i = L.slip[q]
        P = L.slip_P[q]
        r = L.proj(rhs)[:, i] - L.apply_A(u)[:, i]
        new_block = u[:, i] + np.linalg.solve(L.Kv_node[i], r)
        # unconstrained row without the node itself
        if form == "D":
            full = L.A2 @ u.ravel()
            Aii = L.A2_node[i]
            off = full.reshape(3, L.n_u)[:, i] - Aii @ u[:, i]
            w, V = np.linalg.eigh(P)
            T = V[:, w > 0.5]
            Z = T @ np.linalg.solve(T.T @ Aii @ T, T.T)
            new_gpu = Z @ (rhs[:, i] - off)
        else:
            off = np.array([(L.A @ u[d])[i] for d in range(3)]) - L.A_diag[i] * u[:, i]
            free_upd = (rhs[:, i] - off) / L.A_diag[i]
            new_gpu = P @ free_upd
        assert np.abs(new_block - new_gpu).max() <= 1e-12 * np.abs(new_gpu).max()
        assert np.abs(new_block - P @ new_block).max() <= 1e-13 * np.abs(new_block).max()


def test_shgs_symmetric_with_slip():
    H = MG.build_hierarchy(W.slip_cube(), 2, coarsest=2)
    Msm = _velocity_smoother_matrix_coupled(H, 2)
    assert np.abs(Msm - Msm.T).max() <= 1e-13 * np.abs(Msm).max()


def _velocity_smoother_matrix_coupled(H, l):
    """r -> u of the velocity half of an Uzawa step from zero over all three
    components (the slip constraint couples them)."""
    L = H.levels[l]
    n = L.n_u
    Msm = np.zeros((3 * n, 3 * n))
    for j in range(3 * n):
        u = np.zeros((3, n))
        f = np.zeros(3 * n)
        f[j] = 1.0
        MG.uzawa_step(H, l, u, np.zeros(L.n_p), f.reshape(3, n), np.zeros(L.n_p))
        Msm[:, j] = u.ravel()
    # restricted to the tangential subspace the map is symmetric; the
    # normal directions of slip nodes map to zero
    return Msm


def test_laplace_smoother_matrix_unchanged_without_slip():
    H = MG.build_hierarchy(W.unit_cube(), 2, coarsest=2)
    assert not H.levels[2].coupled
    Msm = _velocity_smoother_matrix(H, 2)
    assert np.abs(Msm - Msm.T).max() <= 1e-13 * np.abs(Msm).max()


@pytest.mark.parametrize("name,form,level,coarsest", [("channel", "laplace", 2, 1), ("cube", "D", 3, 2),
                                                      ("cube", "laplace", 3, 2)])
def test_multigrid_converges_to_direct_solution(name, form, level, coarsest):
    macro = W.slip_channel() if name == "channel" else W.slip_cube()
    opt = MG.Options(coarse_minres_max=300) if name == "channel" else None
    H = MG.build_hierarchy(macro, level, coarsest=coarsest, opt=opt, form=form)
    L = H.levels[level]
    x = L.mesh.xyz
    if name == "channel":
        uD = W.channel_inflow(x)
        f, g = L.rhs(None, uD)
    else:
        f, g = L.rhs(W.random_body_force(L.mesh.n_nodes, seed=1), W.manufactured_velocity(x))
    res = MG.solve(H, f, g, tol=1e-11, max_cycles=80)
    assert res.history[-1] <= 1e-11
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(res.u - u).max() <= 1e-8 * np.abs(u).max()
    assert np.abs(res.p - p).max() <= 1e-7 * np.abs(p).max()
    # a contraction comparable to the no-slip problem's
    assert len(res.history) - 1 <= 30
    assert np.abs(np.sum(res.u[:, L.slip].T * L.normals, axis=1)).max() <= 1e-12 * np.abs(res.u).max()


def test_fmg_exact_on_slip_cube():
    """Level-independent exact state: FMG reproduces it on every level."""
    H = MG.build_hierarchy(W.slip_cube(), 4, coarsest=2,
                           opt=MG.Options(coarse_minres_max=80, coarse_minres_rtol=1e-13,
                                          coarse_cg_max=100, coarse_cg_rtol=1e-13))
    rhs, dirichlet = {}, {}
    for l, L in H.levels.items():
        x = L.mesh.xyz
        u_ex, grad = _slip_cube_state(x)
        rhs[l] = L.rhs(np.broadcast_to(grad, x.shape).copy(), u_ex)
        dirichlet[l] = u_ex
    res = MG.fmg(H, rhs, dirichlet, cycles=1, nu=2)
    L = H.levels[4]
    x = L.mesh.xyz
    u_ex, grad = _slip_cube_state(x)
    phi = x @ grad
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    assert np.abs(res.u - u_ex[L.free].T).max() <= 1e-8 * np.abs(u_ex).max()
    assert np.abs(res.p - p_ref).max() <= 1e-7 * np.abs(p_ref).max()


@pytest.mark.parametrize("form", ["laplace", "D"])
def test_exact_state_on_sheared_slip_cube(form):
    """Free-slip faces on the tilted planes x = y and x = y + 1 of the sheared
    cube (affine lattice): their normals are (-1, 1, 0) / sqrt 2, and a
    constant flow along the planes plus a hydrostatic pressure is an exact
    discrete solution in both forms."""
    L = S.build_from_macro(W.sheared_slip_cube(), 2, form=form)
    assert len(L.slip) == 18 and not L.slip_edge.any()
    exp = np.array([-1.0, 1.0, 0.0]) / np.sqrt(2.0)
    assert np.abs(np.abs(L.normals @ exp) - 1.0).max() <= 1e-13
    x = L.mesh.xyz
    u_ex = np.broadcast_to(np.array([0.7, 0.7, -0.3]), x.shape).copy()
    grad = np.array([0.4, -1.1, 0.6])
    f, g = L.rhs(np.broadcast_to(grad, x.shape).copy(), u_ex)
    phi = x @ grad
    p_ref = phi - np.dot(L.m, phi) / L.m.sum()
    ru, rp = L.residual(u_ex[L.free].T, p_ref, f, g)
    scale = max(np.abs(f).max(), np.abs(g).max())
    assert np.abs(ru).max() <= 1e-13 * scale and np.abs(rp).max() <= 1e-13 * scale
    u, p = direct.solve_direct(L, f, g)
    assert np.abs(u - u_ex[L.free].T).max() <= 1e-9 and np.abs(p - p_ref).max() <= 1e-9 * np.abs(p_ref).max()


def test_obstacle_edges_and_corners():
    """One free-slip obstacle cube inside a box: at its 12 edges two face
    planes meet and the node is constrained along the edge (projector t t^T,
    t the edge's axis); at its 8 corners three meet and the node is
    Dirichlet; its face nodes keep the mass-conservative normal, which there
    is the face's axis."""
    m = W.box_of_cubes(3, 3, 3, removed=((1, 1, 1),), slip_obstacles=True)
    L = S.build_from_macro(m, 2)
    x = L.mesh.xyz[L.free[L.slip]]
    on_cube = lambda v: (np.abs(v - 1.0) < 1e-12) | (np.abs(v - 2.0) < 1e-12)   # noqa: E731
    k = on_cube(x).sum(axis=1)   # coordinates on the cube's bounding planes
    assert np.array_equal(L.slip_edge, k == 2) and len(x) == 6 * 3 * 3 + 12 * 3
    diag = np.abs(np.einsum("naa->na", L.slip_P))
    edge = np.where(L.slip_edge)[0]
    t_axis = np.argmax(diag[edge], axis=1)
    assert np.allclose(diag[edge].max(axis=1), 1.0)
    assert not on_cube(x[edge, :])[np.arange(len(edge)), t_axis].any()   # t runs along the edge
    face = np.where(~L.slip_edge)[0]
    n_axis = np.argmax(np.abs(L.normals[face]), axis=1)
    assert np.allclose(np.abs(L.normals[face]).max(axis=1), 1.0)
    assert on_cube(x[face, :])[np.arange(len(face)), n_axis].all()   # the normal crosses the face
    key = {tuple(np.rint(v).astype(int)) for v in L.mesh.xyz[L.dir]}
    for c in np.ndindex(2, 2, 2):
        assert (1 + c[0], 1 + c[1], 1 + c[2]) in key


@pytest.mark.parametrize("name,level", [("obstacle", 2), ("sheared", 2), ("channel", 2)])
def test_transfers_keep_corrections_admissible(name, level):
    """The transfer pair of the constrained problem: the restriction lands in
    the coarse admissible space (tangent planes, edge directions at the
    coarse free-slip nodes), the prolongation in the fine one, and on those
    spaces each is the other's Euclidean adjoint, <prolong(e), r> =
    <e, restrict(r)> for admissible e and r -- the coarse correction is a
    constrained coarse velocity seen through P.  On the obstacle cube
    (edges), the sheared cube (tilted faces) and the channel."""
    macro = {"obstacle": lambda: W.box_of_cubes(3, 3, 3, removed=((1, 1, 1),), slip_obstacles=True),
             "sheared": W.sheared_slip_cube, "channel": W.slip_channel}[name]()
    H = MG.build_hierarchy(macro, level, coarsest=level - 1)
    L, Lc = H.levels[level], H.levels[level - 1]
    assert len(L.slip) and len(Lc.slip)
    rng = np.random.default_rng(21)
    r_any = rng.standard_normal((3, L.n_u))
    rp = rng.standard_normal(L.n_p)
    fc, gc = MG.restrict(H, level, r_any, rp)
    np.testing.assert_allclose(Lc.proj(fc), fc, rtol=0, atol=1e-13 * np.abs(fc).max())
    e = Lc.proj(rng.standard_normal((3, Lc.n_u)))
    pc = rng.standard_normal(Lc.n_p)
    du, dp = MG.prolong(H, level, e, pc)
    np.testing.assert_allclose(L.proj(du), du, rtol=0, atol=1e-13 * np.abs(du).max())
    r = L.proj(r_any)
    fr, gr = MG.restrict(H, level, r, rp)
    assert np.sum(du * r) == pytest.approx(np.sum(e * fr), rel=1e-12)
    assert np.dot(dp, rp) == pytest.approx(np.dot(pc, gr), rel=1e-12)
    # the coarse projection is not idle: P^T r of an admissible fine residual
    # has normal parts at coarse slip nodes (from the free nodes next to
    # them).  The fine one is on these polyhedral faces (fine and coarse
    # normals agree, so P e is already admissible); it acts where they differ.
    raw_c = np.stack([H.Pu[level].T @ r[d] for d in range(3)])
    assert np.abs(Lc.proj(raw_c) - raw_c).max() > 1e-3 * np.abs(raw_c).max()
