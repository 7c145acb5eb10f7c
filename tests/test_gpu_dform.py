"""GPU D-operator formulation (Sec. 2.1, a_2 = 2 nu <D(u), D(v)>) against the
oracle's D form, element by element through the C ABI: operator, right-hand
side with the coupled Dirichlet lift, Uzawa steps with the node-block
smoother (FP64 1e-11, FP32 1e-5), coarse solve with CG on the coupled block,
V-cycle iterates, and whole FP64 and FP32+IR solves."""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG
from tests.helpers import lattice_index, macro_by_name, rel_err, u_from_lattice, u_to_lattice, p_from_lattice, p_to_lattice
from tests.test_gpu_parity import TOL32, TOL64, _load, _p_err, _random_state, _read_up

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


def _pair_d(pkg, name, finest, coarsest, mx=5):
    macro = macro_by_name(name)
    mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, finest, coarsest_level=coarsest,
                    coarse_minres_max=mx, operator_form=1)
    H = MG.build_hierarchy(macro, finest, coarsest=coarsest, opt=MG.Options(coarse_minres_max=mx), form="D")
    return macro, mesh, H


def _data(name, x):
    if name == "cube":
        return W.manufactured_forcing(x), W.manufactured_velocity(x)
    if name == "channel":
        return np.zeros_like(x), W.channel_inflow(x)
    return np.cos(3 * x) + 0.5, 0.2 * np.sin(2 * x)


@pytest.mark.parametrize("name,level", [("cube", 3), ("channel", 2), ("partial", 3)])
def test_operator_rhs_and_smoother(pkg, name, level):
    macro, mesh, H = _pair_d(pkg, name, level, min(2, level - 1))
    L = H.levels[level]
    dims = mesh.dims()
    lat = lattice_index(L, dims)
    u, p, _, _ = _random_state(H, level, 41)
    ku, kp = mesh.apply_operator(u_to_lattice(L, dims, u), p_to_lattice(L, dims, p))
    ou, op = L.apply(u, p)
    assert rel_err(u_from_lattice(L, dims, ku), ou) < TOL64
    assert rel_err(p_from_lattice(L, dims, kp), op) < TOL64
    x = mesh.node_coords()
    fn, ud = _data(name, x)
    mesh.set_rhs(fn, ud)
    f, g = L.rhs(fn[lat], ud[lat])
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "F")), f) < TOL64
    assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "G")), g) < TOL64
    st = _random_state(H, level, 43)
    for prec, tol in ((0, 1e-11), (1, TOL32)):
        _load(mesh, H, level, st, precision=prec)
        mesh.level_op(level, "uzawa_step", precision=prec, count=3)
        uu, pp, ff, gg = (a.copy() for a in st)
        for _ in range(3):
            MG.uzawa_step(H, level, uu, pp, ff, gg)
        gu, gp = _read_up(mesh, H, level, precision=prec)
        assert rel_err(gu, uu) < tol and rel_err(gp, pp) < tol, prec
        mesh.level_op(level, "residual", precision=prec)
        ru, rp = L.residual(uu, pp, ff, gg)
        assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU", prec)), ru) < 10 * tol
        assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "RP", prec)), rp) < 10 * tol
    mesh.close()


@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 4, 2, 5), ("channel", 2, 1, 30), ("partial", 3, 1, 30)])
def test_coarse_solve_and_vcycle_iterates(pkg, name, level, coarsest, mx):
    macro, mesh, H = _pair_d(pkg, name, level, coarsest, mx)
    Lc = H.levels[coarsest]
    stc = _random_state(H, coarsest, 45)
    _load(mesh, H, coarsest, stc)
    mesh.level_op(coarsest, "coarse_solve")
    u, p, f, g = (a.copy() for a in stc)
    MG.vcycle(H, coarsest, u, p, f, g)
    gu, gp = _read_up(mesh, H, coarsest)
    assert rel_err(gu, u) < 1e-9 and _p_err(Lc, gp, p) < 1e-9
    L = H.levels[level]
    st = _random_state(H, level, 47)
    _load(mesh, H, level, st)
    u, p, f, g = (a.copy() for a in st)
    tol = TOL64 if mx <= 5 else 1e-9
    for cyc in range(2):
        mesh.level_op(level, "vcycle")
        MG.vcycle(H, level, u, p, f, g)
        gu, gp = _read_up(mesh, H, level)
        assert rel_err(gu, u) < tol and _p_err(L, gp, p) < tol, cyc
    mesh.close()


@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 4, 2, 5), ("channel", 3, 1, 200)])
def test_d_form_solves_match_oracle(pkg, name, level, coarsest, mx):
    macro, mesh, H = _pair_d(pkg, name, level, coarsest, mx)
    L = H.levels[level]
    dims = mesh.dims()
    lat = lattice_index(L, dims)
    x = mesh.node_coords()
    fn, ud = _data(name, x)
    f, g = L.rhs(fn[lat], ud[lat])
    tight = MG.solve(H, f, g, tol=1e-12, max_cycles=60)
    loose = MG.solve(H, f, g, tol=1e-8, max_cycles=40)
    mesh.set_rhs(fn, ud)
    u, p, st = mesh.solve(tol=1e-12, max_cycles=60, mode=pkg.MODE_FP64)
    assert st.status == 0 and st.cycles == tight.cycles
    np.testing.assert_allclose(st.history, tight.history, rtol=1e-6, atol=1e-13)
    ut = L.scatter(tight.u, ud[lat])
    assert rel_err(u[lat], ut) < 1e-9 and rel_err(p[lat], tight.p) < 1e-8
    eu64 = rel_err(L.scatter(loose.u, ud[lat]), ut)
    ep64 = rel_err(loose.p, tight.p)
    mesh.set_rhs(fn, ud)
    u32, p32, s32 = mesh.solve(tol=1e-8, max_cycles=40, mode=pkg.MODE_FP32_IR)
    assert s32.status == 0 and s32.rel_residual <= 1e-8
    assert rel_err(u32[lat], ut) <= 10 * eu64 + 1e-9
    assert rel_err(p32[lat], tight.p) <= 10 * ep64 + 1e-7
    mesh.close()
