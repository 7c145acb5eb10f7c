"""The oracle on lattice windows (tests.helpers.LatticeWindow) against the
oracle on the whole domain: the device the full-size GPU parity tests use
to have the oracle compute sampled outputs of a level it cannot assemble
(the cube at level 9 has 1.35e8 nodes, the channel at level 6 6.8e7).  The
unit cube at level 6 and a 4 x 4 x 3 box of cubes with two obstacles that
share an edge, no-slip walls, inflow data and do-nothing outflow at level 4
are assembled whole too, and on windows of 33^3 nodes, touching the
boundary, an obstacle, the outflow face or nothing:
  * the right-hand side (random body force, Dirichlet data on the walls)
    at the window's free nodes, g up to a constant (the mean removal of a
    pure Dirichlet window), and the residual rows are the domain's;
  * restriction to the coarse nodes inside the window and prolongation to
    every fine node of the window are the cube's;
  * after one Uzawa step with the window's boundary held, the nodes at
    least 12 lattice steps from a held face (one step per colour phase:
    4 forward, 4 backward velocity colours, 4 pressure colours) carry the
    cube's values."""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG
from tests.helpers import LatticeWindow, rel_err

LEVEL, WL = 6, 5
DIM = (1 << LEVEL) + 1
ORIGINS = [(0, 0, 0), (32, 32, 32), (16, 20, 24), (0, 12, 32)]
PHASES = 12


@pytest.fixture(scope="module")
def cube():
    H = MG.build_hierarchy(W.unit_cube(), LEVEL, coarsest=LEVEL - 1)
    L = H.levels[LEVEL]
    rng = np.random.default_rng(5)
    u, p = rng.standard_normal((3, L.n_u)), rng.standard_normal(L.n_p)
    f, g = rng.standard_normal((3, L.n_u)), rng.standard_normal(L.n_p)
    return H, (u, p, f, g)


def _order(L, dim):
    """Oracle node of each lattice index."""
    lat = L.mesh.ijk[:, 0] + dim * (L.mesh.ijk[:, 1] + dim * L.mesh.ijk[:, 2])
    inv = np.full(dim ** 3, -1)
    inv[lat] = np.arange(len(lat))
    return inv


def _nodal(L, v):
    """(3, n_free) free values -> (n, 3) with zeros on Dirichlet nodes."""
    out = np.zeros((L.n_p, 3))
    out[L.free] = np.asarray(v).T
    return out


@pytest.mark.parametrize("origin", ORIGINS)
def test_window_residual_and_transfers_are_the_cubes(cube, origin):
    H, (u, p, f, g) = cube
    L = H.levels[LEVEL]
    win = LatticeWindow(LEVEL, origin, WL)
    at = _order(L, DIM)[win.index]
    assert np.all(at >= 0)
    np.testing.assert_allclose(win.L.mesh.xyz, L.mesh.xyz[at], rtol=0, atol=1e-15)
    un, fn = _nodal(L, u), _nodal(L, f)
    ru, rp = L.residual(u, p, f, g)
    wru, wrp = win.residual(un[at], p[at], fn[at], g[at])
    inner = ~np.isin(np.arange(len(at)), win.L.dir)
    assert rel_err(wru.T, _nodal(L, ru)[at][win.free]) < 1e-13
    assert rel_err(wrp[inner], rp[at][inner]) < 1e-13
    # restriction to the coarse nodes inside the window, prolongation to all of its fine nodes
    Lc = H.levels[LEVEL - 1]
    cw = LatticeWindow(LEVEL - 1, tuple(o // 2 for o in origin), WL - 1)
    atc = _order(Lc, (DIM + 1) // 2)[cw.index]
    P = MG.prolongation(win.L, cw.L)
    r_full = _nodal(L, ru)[at]
    r_full[win.L.dir] = 0.0
    rp_full = np.where(inner, wrp, 0.0)
    fc = np.stack([H.Pu[LEVEL].T @ ru[d] for d in range(3)])
    gc = H.P[LEVEL].T @ rp
    cin = cw.free
    assert rel_err((P.T @ r_full)[cin], _nodal(Lc, fc)[atc][cin]) < 1e-13
    assert rel_err((P.T @ rp_full)[cin], gc[atc][cin]) < 1e-13
    rng = np.random.default_rng(6)
    uc, pc = rng.standard_normal((3, Lc.n_u)), rng.standard_normal(Lc.n_p)
    pu = _nodal(L, np.stack([H.Pu[LEVEL] @ uc[d] for d in range(3)]))[at]
    wpu = P @ _nodal(Lc, uc)[atc]
    fine_free = ~win.dirichlet
    assert rel_err(wpu[fine_free], pu[fine_free]) < 1e-14
    assert rel_err(P @ pc[atc], (H.P[LEVEL] @ pc)[at]) < 1e-14


@pytest.mark.parametrize("origin", ORIGINS)
def test_window_uzawa_step_core_is_the_cubes(cube, origin):
    H, (u, p, f, g) = cube
    L = H.levels[LEVEL]
    win = LatticeWindow(LEVEL, origin, WL)
    at = _order(L, DIM)[win.index]
    wu, wp = win.uzawa_step(_nodal(L, u)[at], p[at], _nodal(L, f)[at], g[at])
    u1, p1 = u.copy(), p.copy()
    MG.uzawa_step(H, LEVEL, u1, p1, f, g)
    core = win.held_distance >= PHASES
    core_free = core[win.free]
    assert core_free.sum() >= 9 ** 3
    assert rel_err(wu.T[core_free], _nodal(L, u1)[at][win.free][core_free]) < 1e-13
    assert rel_err(wp[core], p1[at][core]) < 1e-13
    # the bound is needed: next to a held face the window's values differ
    near = (win.held_distance < 4)[win.free]
    assert np.abs(wu.T[near] - _nodal(L, u1)[at][win.free][near]).max() > 1e-3


BOX_LEVEL = 4
BOX_ORIGINS = [(16, 16, 16), (0, 16, 0), (32, 0, 16)]


def _box():
    return W.box_of_cubes(4, 4, 3, removed=((1, 1, 1), (2, 2, 1)), outflow_x_max=True)


@pytest.fixture(scope="module")
def box():
    dom = _box()
    H = MG.build_hierarchy(dom, BOX_LEVEL, coarsest=BOX_LEVEL - 1)
    L = H.levels[BOX_LEVEL]
    rng = np.random.default_rng(8)
    u, p = rng.standard_normal((3, L.n_u)), rng.standard_normal(L.n_p)
    f, g = rng.standard_normal((3, L.n_u)), rng.standard_normal(L.n_p)
    return dom, H, (u, p, f, g)


def _order_box(L, dims):
    ijk = L.mesh.ijk
    lat = ijk[:, 0] + dims[0] * (ijk[:, 1] + dims[1] * ijk[:, 2])
    inv = np.full(int(np.prod(dims)), -1)
    inv[lat] = np.arange(len(lat))
    return inv


@pytest.mark.parametrize("origin", BOX_ORIGINS)
def test_box_windows_with_obstacles_and_outflow(box, origin):
    dom, H, (u, p, f, g) = box
    L = H.levels[BOX_LEVEL]
    win = LatticeWindow(BOX_LEVEL, origin, WL, domain=dom)
    at = _order_box(L, dom.lattice_dims(BOX_LEVEL))[win.index]
    assert np.all(at >= 0)
    np.testing.assert_allclose(win.L.mesh.xyz, L.mesh.xyz[at], rtol=0, atol=1e-15)
    # the window's free velocity nodes are the domain's, off the held faces
    free_dom = np.zeros(L.n_p, bool)
    free_dom[L.free] = True
    inner = win.held_distance >= 1
    assert np.array_equal(~win.dirichlet[inner], free_dom[at][inner])
    assert np.array_equal(np.isin(np.arange(len(at)), win.free), free_dom[at] & inner)
    # right-hand side: random body force, inflow data on x = 0
    x = L.mesh.xyz
    fn = W.random_body_force(L.n_p, seed=3)
    ud = np.where(~free_dom[:, None], W.channel_inflow(x), 0.0)
    fu, gg = L.rhs(fn, ud)
    wfu, wg = win.L.rhs(fn[at], np.where(win.dirichlet[:, None], ud[at], 0.0))
    assert rel_err(wfu.T, _nodal(L, fu)[at][win.free]) < 1e-13
    d = wg[inner] - gg[at][inner]
    assert np.abs(d - d.mean()).max() < 1e-13 * np.abs(gg).max()
    # residual and one Uzawa step
    un, fnl = _nodal(L, u), _nodal(L, f)
    ru, rp = L.residual(u, p, f, g)
    wru, wrp = win.residual(un[at], p[at], fnl[at], g[at])
    assert rel_err(wru.T, _nodal(L, ru)[at][win.free]) < 1e-13
    assert rel_err(wrp[inner], rp[at][inner]) < 1e-13
    wu, wp = win.uzawa_step(un[at], p[at], fnl[at], g[at])
    u1, p1 = u.copy(), p.copy()
    MG.uzawa_step(H, BOX_LEVEL, u1, p1, f, g)
    core = win.held_distance >= PHASES
    cf = core[win.free]
    assert cf.sum() > 0
    assert rel_err(wu.T[cf], _nodal(L, u1)[at][win.free][cf]) < 1e-13
    assert rel_err(wp[core], p1[at][core]) < 1e-13
    # transfers
    Lc = H.levels[BOX_LEVEL - 1]
    cw = LatticeWindow(BOX_LEVEL - 1, tuple(o // 2 for o in origin), WL - 1, domain=dom)
    atc = _order_box(Lc, dom.lattice_dims(BOX_LEVEL - 1))[cw.index]
    P = MG.prolongation(win.L, cw.L)
    r_full = np.zeros((len(at), 3))
    r_full[win.free] = wru.T
    fc = np.stack([H.Pu[BOX_LEVEL].T @ ru[d] for d in range(3)])
    gc = H.P[BOX_LEVEL].T @ rp
    assert rel_err((P.T @ r_full)[cw.free], _nodal(Lc, fc)[atc][cw.free]) < 1e-13
    assert rel_err((P.T @ np.where(inner, wrp, 0.0))[cw.free], gc[atc][cw.free]) < 1e-13
    rng = np.random.default_rng(9)
    uc, pc = rng.standard_normal((3, Lc.n_u)), rng.standard_normal(Lc.n_p)
    pu = _nodal(L, np.stack([H.Pu[BOX_LEVEL] @ uc[d] for d in range(3)]))[at]
    fine_free = free_dom[at]
    assert rel_err((P @ _nodal(Lc, uc)[atc])[fine_free], pu[fine_free]) < 1e-14
    assert rel_err(P @ pc[atc], (H.P[BOX_LEVEL] @ pc)[at]) < 1e-14
