"""The oracle on lattice windows (tests.helpers.LatticeWindow) against the
oracle on the whole cube: the device the full-size GPU parity tests use to
have the oracle compute sampled outputs of a level it cannot assemble
(level 9 has 1.35e8 nodes).  At level 6 the whole cube is assembled too,
and on windows of 33^3 nodes, touching the cube's boundary or not:
  * residual rows at the window's interior nodes are the cube's;
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
    fine_free = ~win.on_cube_boundary
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
