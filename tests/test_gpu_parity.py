"""GPU parity: every step of the CUDA path against the CPU oracle, element by
element, on the same seeded inputs, through the C ABI.

Tolerances (element-wise, relative to the field's maximum):
  * FP64 single operations: 1e-12 (rounding order differs: factored stencils
    vs assembled rows);
  * FP64 whole cycles: 1e-12 where the coarse MINRES runs at most 5
    iterations, 1e-9 where it runs 30+ (its Lanczos recurrence amplifies the
    rounding-order differences of dot products); converged solutions 1e-10;
  * FP32 steps against the FP64 oracle: TOL32 = 1e-5.  A node update sums
    about 20 terms bounded by the field maximum, so one update carries at
    most ~20 u = 1.2e-6 relative error (u = 2^-24), plus the rounding of the
    FP32 inputs (6e-8); the smoother contracts, so a few dependent colour
    phases, a V-cycle included, stay below 1e-5;
  * FP32+IR solutions: within 10x (plus a floor) of the error the FP64 oracle
    itself makes when stopped at the same relative residual, both measured
    against the oracle solved to 1e-13 ("equal accuracy").
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, direct, multigrid as MG
from tests.helpers import (lattice_index, macro_by_name, nodal_to_lattice, p_from_lattice, p_to_lattice,
                           rel_err, u_from_lattice, u_to_lattice)

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


def _pair(pkg, name, finest, coarsest=2, **opt):
    macro = macro_by_name(name)
    mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, finest, coarsest_level=coarsest, **opt)
    oo = MG.Options(**{k: v for k, v in opt.items() if k in MG.Options.__dataclass_fields__})
    H = MG.build_hierarchy(macro, finest, coarsest=coarsest, opt=oo)
    return macro, mesh, H


def _random_state(H, l, seed):
    """Random iterate and right-hand side; on pure-Dirichlet meshes g is made
    consistent (orthogonal to the constant pressure null vector)."""
    L = H.levels[l]
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(L.n_p)
    if L.pure_dirichlet:
        g -= g.mean()
    return (rng.standard_normal((3, L.n_u)), rng.standard_normal(L.n_p),
            rng.standard_normal((3, L.n_u)), g)


def _p_err(L, gp, p):
    """Pressure error modulo the constant null vector of pure-Dirichlet problems
    (a coarse Krylov solve leaves its component undetermined)."""
    if L.pure_dirichlet:
        return rel_err(L.project_pressure(gp), L.project_pressure(p))
    return rel_err(gp, p)


def _load(mesh, H, l, state, precision=0):
    L = H.levels[l]
    dims = mesh.dims(l)
    u, p, f, g = state
    mesh.level_field(l, "U", precision, u_to_lattice(L, dims, u))
    mesh.level_field(l, "P", precision, p_to_lattice(L, dims, p))
    mesh.level_field(l, "F", precision, u_to_lattice(L, dims, f))
    mesh.level_field(l, "G", precision, p_to_lattice(L, dims, g))


def _read_up(mesh, H, l, precision=0):
    L = H.levels[l]
    dims = mesh.dims(l)
    return (u_from_lattice(L, dims, mesh.level_field(l, "U", precision)),
            p_from_lattice(L, dims, mesh.level_field(l, "P", precision)))


# ---- operator and right-hand side ---------------------------------------------------

@pytest.mark.parametrize("name,level", [("cube", 2), ("cube", 4), ("cube", 5), ("channel", 1), ("channel", 2),
                                        ("partial", 3), ("sheared", 3)])
def test_apply_operator(pkg, name, level):
    macro, mesh, H = _pair(pkg, name, level, coarsest=min(2, level))
    L = H.levels[level]
    dims = mesh.dims()
    u, p, _, _ = _random_state(H, level, 1)
    ku, kp = mesh.apply_operator(u_to_lattice(L, dims, u), p_to_lattice(L, dims, p))
    ou, op = L.apply(u, p)
    assert rel_err(u_from_lattice(L, dims, ku), ou) < TOL64
    assert rel_err(p_from_lattice(L, dims, kp), op) < TOL64
    # nothing written off the unknowns
    lat = lattice_index(L, dims)
    mask = np.ones(len(kp), bool)
    mask[lat] = False
    assert np.all(kp[mask] == 0) and np.all(ku[mask] == 0)


@pytest.mark.parametrize("name,level", [("cube", 3), ("cube", 5), ("channel", 2), ("partial", 3), ("sheared", 3)])
def test_set_rhs(pkg, name, level):
    macro, mesh, H = _pair(pkg, name, level, coarsest=min(2, level))
    L = H.levels[level]
    dims = mesh.dims()
    x = mesh.node_coords()
    rng = np.random.default_rng(3)
    fn = rng.standard_normal(x.shape)
    ud = W.manufactured_velocity(x) if name != "channel" else W.channel_inflow(x)
    if name == "sheared":
        np.testing.assert_allclose(x, macro.lattice_coords(level), atol=1e-14)
    mesh.set_rhs(fn, ud)
    lat = lattice_index(L, dims)
    f, g = L.rhs(fn[lat], ud[lat])
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "F")), f) < TOL64
    assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "G")), g) < TOL64


# ---- smoother pieces, transfers, coarse solve ---------------------------------------------

KERNEL_FORMS = [(0, 0), (-1, 1), (-1, 2), (-1, 4), (0, 4)]


@pytest.mark.parametrize("spec,cbz", KERNEL_FORMS)
@pytest.mark.parametrize("name,level", [("cube", 3), ("channel", 2), ("partial", 3), ("sheared", 3)])
def test_smoother_pieces(pkg, name, level, spec, cbz):
    """Smoother steps against the oracle, with the colour sweeps run by the
    grid kernels in the speculative node form of small levels (spec = 0, the
    default here) or the flags-first form of large levels (spec = -1), with
    1, 2 or 4 planes per colour block (cbz; 0 = the level's default)."""
    macro, mesh, H = _pair(pkg, name, level, coarsest=min(2, level), spec_max_nodes=spec, colour_block_z=cbz)
    L = H.levels[level]
    dims = mesh.dims()
    st = _random_state(H, level, 7)
    u, p, f, g = (a.copy() for a in st)
    _load(mesh, H, level, st)
    # RU = F - B^T P
    mesh.level_op(level, "vel_rhs")
    ru = np.stack([f[d] - L.BT[d] @ p for d in range(3)])
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU")), ru) < TOL64
    # forward and backward velocity sweeps with RU as right-hand side
    mesh.level_op(level, "vel_forward")
    for d in range(3):
        MG._gs_sweep(L.A, L.A_diag, u[d], ru[d], H.colours_u[level], (0, 1, 2, 3))
    gu, _ = _read_up(mesh, H, level)
    assert rel_err(gu, u) < TOL64
    mesh.level_op(level, "vel_backward")
    for d in range(3):
        MG._gs_sweep(L.A, L.A_diag, u[d], ru[d], H.colours_u[level], (3, 2, 1, 0))
    gu, _ = _read_up(mesh, H, level)
    assert rel_err(gu, u) < TOL64
    # RP = B U - G, then the relaxed pressure sweep
    mesh.level_op(level, "pres_rhs")
    rp = sum(L.B[d] @ u[d] for d in range(3)) - g
    assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "RP")), rp) < TOL64
    mesh.level_op(level, "pres_sweep")
    MG._gs_sweep(L.C, L.C_diag, p, rp, H.colours_p[level], (0, 1, 2, 3), relax=H.opt.omega)
    _, gp = _read_up(mesh, H, level)
    assert rel_err(gp, p) < TOL64
    # the same sweeps with the right-hand sides formed at each node
    _load(mesh, H, level, st)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(level, "vel_forward_f")
    ru = np.stack([f[d] - L.BT[d] @ p for d in range(3)])
    for d in range(3):
        MG._gs_sweep(L.A, L.A_diag, u[d], ru[d], H.colours_u[level], (0, 1, 2, 3))
    gu, _ = _read_up(mesh, H, level)
    assert rel_err(gu, u) < TOL64
    mesh.level_op(level, "pres_sweep_f")
    rp = sum(L.B[d] @ u[d] for d in range(3)) - g
    MG._gs_sweep(L.C, L.C_diag, p, rp, H.colours_p[level], (0, 1, 2, 3), relax=H.opt.omega)
    _, gp = _read_up(mesh, H, level)
    assert rel_err(gp, p) < TOL64
    # whole Uzawa steps
    _load(mesh, H, level, st)
    mesh.level_op(level, "uzawa_step", count=3)
    u, p, f, g = (a.copy() for a in st)
    for _ in range(3):
        MG.uzawa_step(H, level, u, p, f, g)
    gu, gp = _read_up(mesh, H, level)
    assert rel_err(gu, u) < 1e-11 and rel_err(gp, p) < 1e-11
    # residual
    mesh.level_op(level, "residual")
    ru, rp = L.residual(u, p, f, g)
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU")), ru) < 1e-11
    assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "RP")), rp) < 1e-11


@pytest.mark.parametrize("cbz,fused,pairs", [(1, -1, 0), (2, -1, 0), (2, -1, 1), (1, 1, 0)])
@pytest.mark.parametrize("name,level", [("cube", 4), ("channel", 2), ("partial", 3)])
def test_fp32_steps_match_oracle(pkg, name, level, cbz, fused, pairs):
    """Every FP32 kernel of the V-cycle against the FP64 oracle on the same
    seeded state (written into the FP32 hierarchy, i.e. rounded once):
    forward velocity sweep and pressure sweep with their right-hand sides
    formed at each node, whole Uzawa steps, residual, restriction,
    prolongation and a whole V-cycle rooted at the finest level.  fused = 1
    runs every level's Uzawa steps as the three colour-fused passes; pairs = 1
    has the colour kernels update two nodes per thread (0: the default, one)."""
    macro, mesh, H = _pair(pkg, name, level, coarsest=level - 2, coarse_minres_max=5, spec_max_nodes=-1,
                           colour_block_z=cbz, fused_min_nodes=fused, colour_pairs=pairs)
    L = H.levels[level]
    dims = mesh.dims()
    st = _random_state(H, level, 13)
    # sweeps with the right-hand sides formed at the node
    _load(mesh, H, level, st, precision=1)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(level, "vel_forward_f", precision=1)
    ru = np.stack([f[d] - L.BT[d] @ p for d in range(3)])
    for d in range(3):
        MG._gs_sweep(L.A, L.A_diag, u[d], ru[d], H.colours_u[level], (0, 1, 2, 3))
    gu, _ = _read_up(mesh, H, level, precision=1)
    assert rel_err(gu, u) < TOL32
    mesh.level_op(level, "pres_sweep_f", precision=1)
    rp = sum(L.B[d] @ u[d] for d in range(3)) - g
    MG._gs_sweep(L.C, L.C_diag, p, rp, H.colours_p[level], (0, 1, 2, 3), relax=H.opt.omega)
    _, gp = _read_up(mesh, H, level, precision=1)
    assert rel_err(gp, p) < TOL32
    # whole Uzawa steps, then the residual
    _load(mesh, H, level, st, precision=1)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(level, "uzawa_step", precision=1, count=2)
    for _ in range(2):
        MG.uzawa_step(H, level, u, p, f, g)
    gu, gp = _read_up(mesh, H, level, precision=1)
    assert rel_err(gu, u) < TOL32 and rel_err(gp, p) < TOL32
    mesh.level_op(level, "residual", precision=1)
    ru, rp = L.residual(u, p, f, g)
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU", 1)), ru) < TOL32
    assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "RP", 1)), rp) < TOL32
    # restriction of that residual, prolongation of a random coarse correction
    Lc = H.levels[level - 1]
    dc = mesh.dims(level - 1)
    mesh.level_op(level, "restrict", precision=1)
    ru32 = u_from_lattice(L, dims, mesh.level_field(level, "RU", 1))
    rp32 = p_from_lattice(L, dims, mesh.level_field(level, "RP", 1))
    fc = np.stack([H.Pu[level].T @ ru32[d] for d in range(3)])
    assert rel_err(u_from_lattice(Lc, dc, mesh.level_field(level - 1, "F", 1)), fc) < TOL32
    assert rel_err(p_from_lattice(Lc, dc, mesh.level_field(level - 1, "G", 1)), H.P[level].T @ rp32) < TOL32
    rng = np.random.default_rng(14)
    uc, pc = rng.standard_normal((3, Lc.n_u)), rng.standard_normal(Lc.n_p)
    mesh.level_field(level - 1, "U", 1, u_to_lattice(Lc, dc, uc))
    mesh.level_field(level - 1, "P", 1, p_to_lattice(Lc, dc, pc))
    gu0, gp0 = _read_up(mesh, H, level, precision=1)
    mesh.level_op(level, "prolong_add", precision=1)
    gu, gp = _read_up(mesh, H, level, precision=1)
    assert rel_err(gu, gu0 + np.stack([H.Pu[level] @ uc[d] for d in range(3)])) < TOL32
    assert rel_err(gp, gp0 + H.P[level] @ pc) < TOL32
    # a whole FP32 V-cycle (coarse solve in FP64 on the FP32 residual)
    _load(mesh, H, level, st, precision=1)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(level, "vcycle", precision=1)
    MG.vcycle(H, level, u, p, f, g)
    gu, gp = _read_up(mesh, H, level, precision=1)
    assert rel_err(gu, u) < TOL32 and _p_err(L, gp, p) < TOL32
    mesh.close()


def test_level6_large_level_kernels_match_oracle(pkg):
    """The kernels in the forms the bench uses on its largest levels
    (flags-first node form, two planes per colour block, the residual four
    nodes per thread), on a level large enough to span many blocks with
    ragged edges (65^3 nodes): FP64 Uzawa steps and a V-cycle against the
    oracle, and FP32 Uzawa steps."""
    macro, mesh, H = _pair(pkg, "cube", 6, coarsest=2, spec_max_nodes=-1, colour_block_z=2, quad_min_nodes=1)
    L = H.levels[6]
    st = _random_state(H, 6, 23)
    _load(mesh, H, 6, st)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(6, "uzawa_step", count=2)
    for _ in range(2):
        MG.uzawa_step(H, 6, u, p, f, g)
    gu, gp = _read_up(mesh, H, 6)
    assert rel_err(gu, u) < TOL64 and rel_err(gp, p) < TOL64
    mesh.level_op(6, "vcycle")
    MG.vcycle(H, 6, u, p, f, g)
    gu, gp = _read_up(mesh, H, 6)
    assert rel_err(gu, u) < TOL64 and _p_err(L, gp, p) < TOL64
    _load(mesh, H, 6, st, precision=1)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(6, "uzawa_step", precision=1, count=2)
    for _ in range(2):
        MG.uzawa_step(H, 6, u, p, f, g)
    gu, gp = _read_up(mesh, H, 6, precision=1)
    assert rel_err(gu, u) < TOL32 and rel_err(gp, p) < TOL32
    mesh.close()


@pytest.mark.parametrize("name,level", [("cube", 4), ("cube", 5), ("channel", 2), ("partial", 3), ("sheared", 3)])
def test_quad_residual_matches_oracle(pkg, name, level):
    """The FP32 residual four nodes per thread (quad_min_nodes = 1 forces it
    on every level): quads of regular nodes take the shared-load path, quads
    with a boundary, Dirichlet or outside node the per-node body (the
    partially filled and sheared meshes exercise the fallback), against the
    oracle, and FP32 V-cycles with it; the FP64 residual keeps the per-node
    kernel."""
    macro, mesh, H = _pair(pkg, name, level, coarsest=min(2, level - 1), quad_min_nodes=1)
    L = H.levels[level]
    dims = mesh.dims()
    st = _random_state(H, level, 29)
    ru, rp = L.residual(*st)
    for prec, tol in ((0, TOL64), (1, TOL32)):
        _load(mesh, H, level, st, precision=prec)
        mesh.level_op(level, "residual", precision=prec)
        assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU", prec)), ru) < tol, prec
        assert rel_err(p_from_lattice(L, dims, mesh.level_field(level, "RP", prec)), rp) < tol, prec
    _load(mesh, H, level, st, precision=1)
    u, p, f, g = (a.copy() for a in st)
    mesh.level_op(level, "vcycle", precision=1)
    MG.vcycle(H, level, u, p, f, g)
    gu, gp = _read_up(mesh, H, level, precision=1)
    assert rel_err(gu, u) < TOL32 and _p_err(L, gp, p) < TOL32
    mesh.close()


@pytest.mark.parametrize("rows", [0, 1, 3])
@pytest.mark.parametrize("name,level", [("cube", 5), ("channel", 3), ("partial", 4)])
def test_fused_passes_match_grid_kernels_and_oracle(pkg, name, level, rows):
    """The colour-fused FP32 passes (every level fused; rows = tile rows, 0 =
    the per-level choice, 1 and 3 give many ragged tiles) evaluate the same
    per-node expressions as the per-colour grid kernels: Uzawa steps agree to
    FP32 rounding (only the compiler's contraction into fused multiply-adds
    may differ) and with the FP64 oracle at TOL32; each pass alone moves its
    fields as documented (pass 0 leaves U, P and writes RU)."""
    macro = macro_by_name(name)
    H = MG.build_hierarchy(macro, level, coarsest=level - 1)
    L = H.levels[level]
    dims_mesh = [pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, level, coarsest_level=level - 1,
                          fused_min_nodes=fz, fused_tile_rows=rows) for fz in (-1, 1)]
    st = _random_state(H, level, 17)
    outs = []
    for mesh in dims_mesh:
        _load(mesh, H, level, st, precision=1)
        mesh.level_op(level, "uzawa_step", precision=1, count=2)
        outs.append(_read_up(mesh, H, level, precision=1))
    assert rel_err(outs[1][0], outs[0][0]) < 1e-6
    assert rel_err(outs[1][1], outs[0][1]) < 1e-6
    u, p, f, g = (a.copy() for a in st)
    for _ in range(2):
        MG.uzawa_step(H, level, u, p, f, g)
    assert rel_err(outs[1][0], u) < TOL32 and rel_err(outs[1][1], p) < TOL32
    # pass 0 alone: the forward velocity sweep lands in RU, U and P untouched
    mesh = dims_mesh[1]
    dims = mesh.dims()
    _load(mesh, H, level, st, precision=1)
    u0, p0 = _read_up(mesh, H, level, precision=1)
    mesh.level_op(level, "fused_pass0", precision=1)
    u, p, f, g = (a.copy() for a in st)
    ru = np.stack([f[d] - L.BT[d] @ p for d in range(3)])
    for d in range(3):
        MG._gs_sweep(L.A, L.A_diag, u[d], ru[d], H.colours_u[level], (0, 1, 2, 3))
    assert rel_err(u_from_lattice(L, dims, mesh.level_field(level, "RU", 1)), u) < TOL32
    gu, gp = _read_up(mesh, H, level, precision=1)
    assert np.array_equal(gu, u0) and np.array_equal(gp, p0)
    for mesh in dims_mesh:
        mesh.close()


def test_fused_pass_wait_timeout(pkg):
    """A fused pass whose bounded mbarrier wait runs out reports HHG_ECUDA
    without faulting.  The test option announces 16 bytes more than the first
    staged plane delivers, so that wait cannot complete (1024 polls); the CTA
    withdraws the excess, waits for its valid copies to land and returns.  The
    error word is cleared: the next call on the same mesh that runs no fused
    pass succeeds, and a mesh without the option still matches the grid
    kernels."""
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 5, fused_min_nodes=1, wait_poll_limit=1024,
                    fused_wait_test=1)
    H = MG.build_hierarchy(cube, 5, coarsest=4)
    st = _random_state(H, 5, 31)
    _load(mesh, H, 5, st, precision=1)
    with pytest.raises(pkg.HHGError) as e:
        mesh.level_op(5, "uzawa_step", precision=1)
    assert e.value.code == -6 and "gave up waiting" in str(e.value)
    mesh.level_op(5, "uzawa_step", precision=0)   # grid kernels: no stale error
    good = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 5, fused_min_nodes=1)
    ref = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 5, fused_min_nodes=-1)
    outs = []
    for m in (good, ref):
        _load(m, H, 5, st, precision=1)
        m.level_op(5, "uzawa_step", precision=1)
        outs.append(_read_up(m, H, 5, precision=1))
    assert rel_err(outs[0][0], outs[1][0]) < 1e-6 and rel_err(outs[0][1], outs[1][1]) < 1e-6
    for m in (mesh, good, ref):
        m.close()


@pytest.mark.parametrize("name,level", [("cube", 4), ("channel", 2), ("partial", 3), ("sheared", 3)])
def test_transfers(pkg, name, level):
    macro, mesh, H = _pair(pkg, name, level, coarsest=level - 1)
    Lf, Lc = H.levels[level], H.levels[level - 1]
    df, dc = mesh.dims(level), mesh.dims(level - 1)
    rng = np.random.default_rng(11)
    ru = rng.standard_normal((3, Lf.n_u))
    rp = rng.standard_normal(Lf.n_p)
    mesh.level_field(level, "RU", 0, u_to_lattice(Lf, df, ru))
    mesh.level_field(level, "RP", 0, p_to_lattice(Lf, df, rp))
    mesh.level_op(level, "restrict")
    fc = np.stack([H.Pu[level].T @ ru[d] for d in range(3)])
    gc = H.P[level].T @ rp
    assert rel_err(u_from_lattice(Lc, dc, mesh.level_field(level - 1, "F")), fc) < TOL64
    assert rel_err(p_from_lattice(Lc, dc, mesh.level_field(level - 1, "G")), gc) < TOL64
    assert np.all(mesh.level_field(level - 1, "U") == 0)
    # prolongate a random coarse correction onto a random fine iterate
    uc = rng.standard_normal((3, Lc.n_u))
    pc = rng.standard_normal(Lc.n_p)
    uf = rng.standard_normal((3, Lf.n_u))
    pf = rng.standard_normal(Lf.n_p)
    mesh.level_field(level - 1, "U", 0, u_to_lattice(Lc, dc, uc))
    mesh.level_field(level - 1, "P", 0, p_to_lattice(Lc, dc, pc))
    mesh.level_field(level, "U", 0, u_to_lattice(Lf, df, uf))
    mesh.level_field(level, "P", 0, p_to_lattice(Lf, df, pf))
    mesh.level_op(level, "prolong_add")
    gu, gp = _read_up(mesh, H, level)
    assert rel_err(gu, uf + np.stack([H.Pu[level] @ uc[d] for d in range(3)])) < TOL64
    assert rel_err(gp, pf + H.P[level] @ pc) < TOL64


@pytest.mark.parametrize("name,level,mx", [("cube", 2, 5), ("cube", 3, 30), ("channel", 0, 40), ("partial", 2, 30)])
def test_coarse_solve(pkg, name, level, mx):
    macro, mesh, H = _pair(pkg, name, level, coarsest=level, coarse_minres_max=mx)
    L = H.levels[level]
    st = _random_state(H, level, 5)
    _load(mesh, H, level, st)
    mesh.level_op(level, "coarse_solve")
    u, p, f, g = (a.copy() for a in st)
    MG.vcycle(H, level, u, p, f, g)   # on the coarsest level: the MINRES correction
    gu, gp = _read_up(mesh, H, level)
    # rounding differences are amplified by the Krylov recurrence; 1e-9 is
    # far below the 5e-3 tolerance the solver is asked for
    assert rel_err(gu, u) < 1e-9 and _p_err(L, gp, p) < 1e-9


# ---- cycles and solves ------------------------------------------------------------------------

@pytest.mark.parametrize("spec,cbz", KERNEL_FORMS)
@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 3, 2, 5), ("cube", 5, 2, 5), ("channel", 2, 1, 200),
                                                    ("partial", 3, 1, 30), ("sheared", 4, 2, 5)])
def test_vcycle_iterates(pkg, name, level, coarsest, mx, spec, cbz):
    macro, mesh, H = _pair(pkg, name, level, coarsest=coarsest, coarse_minres_max=mx, spec_max_nodes=spec,
                           colour_block_z=cbz)
    L = H.levels[level]
    st = _random_state(H, level, 9)
    _load(mesh, H, level, st)
    u, p, f, g = (a.copy() for a in st)
    tol = TOL64 if mx <= 5 else 1e-9
    for cyc in range(2):
        mesh.level_op(level, "vcycle")
        MG.vcycle(H, level, u, p, f, g)
        gu, gp = _read_up(mesh, H, level)
        print(name, level, "cycle", cyc, "u err", rel_err(gu, u), "p err", _p_err(L, gp, p))
        assert rel_err(gu, u) < tol, cyc
        assert _p_err(L, gp, p) < tol, cyc


@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 4, 2, 5), ("cube", 5, 2, 5), ("channel", 3, 1, 200),
                                                    ("sheared", 4, 2, 5)])
def test_fp64_solve_matches_oracle(pkg, name, level, coarsest, mx):
    macro, mesh, H = _pair(pkg, name, level, coarsest=coarsest, coarse_minres_max=mx)
    L = H.levels[level]
    dims = mesh.dims()
    x = mesh.node_coords()
    lat = lattice_index(L, dims)
    if name in ("cube", "sheared"):
        fn, ud = W.manufactured_forcing(x), W.manufactured_velocity(x)
    else:
        fn, ud = np.zeros_like(x), W.channel_inflow(x)
    mesh.set_rhs(fn, ud)
    u, p, st = mesh.solve(tol=1e-10, max_cycles=40, mode=pkg.MODE_FP64)
    f, g = L.rhs(fn[lat], ud[lat])
    ref = MG.solve(H, f, g, tol=1e-10, max_cycles=40, keep_iterates=False)
    assert st.status == 0 and st.cycles == ref.cycles
    # relative residuals near 1e-10 sit at the rounding floor of a residual
    # assembled from O(1) terms: compare with an absolute floor
    np.testing.assert_allclose(st.history, ref.history, rtol=1e-7, atol=1e-14)
    uo = L.scatter(ref.u, ud[lat])
    assert rel_err(u[lat], uo) < 1e-10
    assert rel_err(p[lat], ref.p) < 1e-10
    if name in ("cube", "sheared"):
        m = L.m
        assert abs(np.dot(m, p[lat])) < 1e-12 * np.abs(p).max()


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 5, 2, 5), ("channel", 3, 1, 200)])
def test_fp32_ir_solve(pkg, name, level, coarsest, mx, fused):
    """FP32 V-cycles inside FP64 refinement reach the FP64 tolerance, and the
    solution's error against the oracle (solved to 1e-13) is within 10x of
    the error the FP64 oracle itself makes when stopped at the same relative
    residual (plus a floor of 1e-9 for u, 1e-7 for p, relative to the field
    maxima).  The GPU FP64 solve is checked the same way."""
    macro, mesh, H = _pair(pkg, name, level, coarsest=coarsest, coarse_minres_max=mx, fused_min_nodes=fused)
    L = H.levels[level]
    dims = mesh.dims()
    x = mesh.node_coords()
    lat = lattice_index(L, dims)
    if name == "cube":
        fn, ud = W.manufactured_forcing(x), W.manufactured_velocity(x)
    else:
        fn, ud = np.zeros_like(x), W.channel_inflow(x)
    f, g = L.rhs(fn[lat], ud[lat])
    tight = MG.solve(H, f, g, tol=1e-13, max_cycles=80)
    loose = MG.solve(H, f, g, tol=1e-8, max_cycles=40)
    ut = L.scatter(tight.u, ud[lat])
    eu64 = rel_err(L.scatter(loose.u, ud[lat]), ut)
    ep64 = rel_err(loose.p, tight.p)
    for mode in (pkg.MODE_FP32_IR, pkg.MODE_FP64):
        mesh.set_rhs(fn, ud)
        u, p, st = mesh.solve(tol=1e-8, max_cycles=40, mode=mode)
        assert st.status == 0 and st.rel_residual <= 1e-8
        eu = rel_err(u[lat], ut)
        ep = rel_err(p[lat], tight.p)
        print(name, level, "mode", mode, "cycles", st.cycles, "oracle", loose.cycles, "err u", eu, "vs", eu64,
              "err p", ep, "vs", ep64)
        assert eu <= 10 * eu64 + 1e-9, (eu, eu64)
        assert ep <= 10 * ep64 + 1e-7, (ep, ep64)


@pytest.mark.parametrize("name,level,coarsest,mx", [("cube", 5, 2, 5), ("channel", 3, 1, 200), ("partial", 4, 1, 30)])
def test_fixed_point_refinement_residual(pkg, name, level, coarsest, mx):
    """FP32+IR with the refinement residual's regular-node stencils in 64-bit
    fixed point against the same solve with the residual in FP64: the same
    cycle count, relative residual histories equal to 1e-6 relative or 1e-12
    absolute, and solutions equal far below the solver tolerance."""
    macro = macro_by_name(name)
    outs = []
    for fx in (0, 1):
        mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, level, coarsest_level=coarsest,
                        coarse_minres_max=mx, ir_fixed_point=fx)
        x = mesh.node_coords()
        if name == "cube":
            fn, ud = W.manufactured_forcing(x), W.manufactured_velocity(x)
        else:
            fn, ud = W.random_body_force(x.shape[0]), W.channel_inflow(x) if name == "channel" else np.zeros_like(x)
        mesh.set_rhs(fn, ud)
        u, p, st = mesh.solve(tol=1e-10, max_cycles=60, mode=pkg.MODE_FP32_IR)
        assert st.status == 0
        outs.append((u, p, st))
        mesh.close()
    (u0, p0, s0), (u1, p1, s1) = outs
    assert s0.cycles == s1.cycles
    # below 1e-10 the histories differ by the rounding of the two residual
    # evaluations (4.5e-14 absolute seen on the partial mesh)
    np.testing.assert_allclose(s1.history, s0.history, rtol=1e-6, atol=1e-12)
    assert rel_err(u1, u0) < 1e-9 and rel_err(p1, p0) < 1e-8
    # from a zero iterate the first cycle updates in FP64 (a zero field has
    # no scale for its correction); no cycle needs its update redone
    assert s0.fx_rescales == 0 and s1.fx_rescales == 0


def test_fixed_point_rescaling(pkg):
    """The fixed-point iterate's checks: an initial iterate 1e-6 times the
    solution makes the first correction too large for its scales (the update
    is redone in FP64 and rescaled), 1.01 times the solution needs no
    rescaling; both solves follow the FP64-iterate solve."""
    cube = W.unit_cube()
    meshes = {fx: pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 4, ir_fixed_point=fx) for fx in (0, 1)}
    x = meshes[0].node_coords()
    for m in meshes.values():
        m.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    us, ps, _ = meshes[0].solve(tol=1e-11, max_cycles=60, mode=pkg.MODE_FP32_IR)
    for scale, rescales in ((1e-6, 1), (1.01, 0)):
        outs = {}
        for fx, m in meshes.items():
            m.set_initial(scale * us, scale * ps)
            outs[fx] = m.solve(tol=1e-9, max_cycles=60, mode=pkg.MODE_FP32_IR)
        (u0, p0, s0), (u1, p1, s1) = outs[0], outs[1]
        assert s0.status == 0 and s1.status == 0 and s0.cycles == s1.cycles
        assert s1.fx_rescales == rescales
        np.testing.assert_allclose(s1.history, s0.history, rtol=1e-6, atol=1e-12)
        assert rel_err(u1, u0) < 1e-9 and rel_err(p1, p0) < 1e-8
    for m in meshes.values():
        m.close()


def test_edge_cases(pkg):
    cube = W.unit_cube()
    # finest == coarsest: the solve is the coarse MINRES alone
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 2, coarsest_level=2, coarse_minres_max=200,
                    coarse_minres_rtol=1e-12, coarse_cg_rtol=1e-14, coarse_cg_max=100)
    x = mesh.node_coords()
    mesh.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    u, p, st = mesh.solve(tol=1e-9, max_cycles=20)
    assert st.status == 0
    H = MG.build_hierarchy(cube, 2)
    L = H.levels[2]
    lat = lattice_index(L, mesh.dims())
    f, g = L.rhs(W.manufactured_forcing(L.mesh.xyz), W.manufactured_velocity(L.mesh.xyz))
    ud, pd = direct.solve_direct(L, f, g)
    assert rel_err(u[lat][L.free].T, ud) < 1e-8
    mesh.close()
    # zero right-hand side: nothing to do, zero solution
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 3)
    mesh.set_rhs(None, None)
    u, p, st = mesh.solve(tol=1e-8, max_cycles=10)
    assert st.cycles == 0 and np.all(u == 0) and np.all(p == 0)
    # call order
    mesh2 = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 3)
    with pytest.raises(pkg.HHGError) as e:
        mesh2.solve()
    assert e.value.code == -7
    # coarsest level 0 hierarchy (deepest cycle)
    mesh3 = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 4, coarsest_level=0, coarse_minres_max=50)
    x = mesh3.node_coords()
    mesh3.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    _, _, st = mesh3.solve(tol=1e-8, max_cycles=30)
    assert st.status == 0


def test_paper_protocol_random_guess(pkg, golden):
    """f = 0, u0 ~ U[0,1], p0 ~ U[0, 1/h_min] (Sec. 3.6), level 4 = paper L = 2:
    GPU and oracle take the same number of cycles (paper: 9)."""
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 4)
    H = MG.build_hierarchy(cube, 4)
    L = H.levels[4]
    dims = mesh.dims()
    lat = lattice_index(L, dims)
    h_min = (L.mesh.h ** 3 / 6.0) ** (1.0 / 3.0)
    u0, p0 = W.random_initial_guess(mesh.num_nodes(), h_min, seed=0)
    mesh.set_rhs(None, None)
    mesh.set_initial(u0, p0)
    _, _, st = mesh.solve(tol=1e-8, max_cycles=30)
    f, g = L.rhs(None, None)
    ref = MG.solve(H, f, g, u0=u0[lat][L.free].T, p0=p0[lat], tol=1e-8, max_cycles=30)
    assert st.cycles == ref.cycles
    assert abs(st.cycles - golden["itertime1_umg"]["rows"][0]["iter"]) <= 2


# ---- adjoint ---------------------------------------------------------------------------------

def test_adjoint_gradient_matches_oracle(pkg):
    ch = W.obstacle_channel()
    level = 2
    mesh = pkg.Mesh(ch.vertices, ch.tets, ch.bc_flags, level, coarsest_level=1, coarse_minres_max=300)
    L = MG.build_hierarchy(ch, level, coarsest=1).levels[level]
    dims = mesh.dims()
    lat = lattice_index(L, dims)
    x = mesh.node_coords()
    psi = W.outflow_flux_weight(x)
    w = mesh.outflow_weights()
    np.testing.assert_allclose(w[lat], L.ops.w_out, atol=1e-14)
    mesh.set_rhs(None, W.channel_inflow(x))
    mesh.solve(tol=1e-10, max_cycles=40)
    grad, st = mesh.adjoint_gradient(ju=w * psi[:, None], tol=1e-12, max_cycles=80)
    ref = adjoint.gradient_direct(L, psi[lat])
    assert rel_err(grad[lat], ref) < 1e-9
    # the forward iterate is left untouched
    u2, _ = mesh.get_solution()
    u1, _, _ = mesh.solve(tol=1e-10, max_cycles=0)
    assert np.array_equal(u1, u2)


FUSED = {"block": dict(fuse_coarse_levels=1),
         "cluster16": dict(fuse_coarse_levels=1, fuse_max_nodes=1 << 16, team_blocks=16),
         "cluster4": dict(fuse_coarse_levels=1, fuse_max_nodes=1 << 16, team_blocks=4),
         "resident16": dict(fuse_coarse_levels=2, team_blocks=16),
         "resident8": dict(fuse_coarse_levels=2, team_blocks=8),
         "resident8_flagtests": dict(fuse_coarse_levels=2, team_blocks=8, resident_node_lists=-1)}


@pytest.mark.parametrize("fused", sorted(FUSED))
@pytest.mark.parametrize("name,level,coarsest", [("cube", 5, 2), ("cube", 3, 2), ("channel", 2, 0), ("partial", 3, 1)])
def test_fused_coarse_levels_match_per_level_kernels(pkg, name, level, coarsest, fused):
    """The fused cycle of the coarse levels (one block, a thread-block
    cluster, or levels resident in a cluster's shared memory) does the same
    arithmetic as the per-level kernels (FP64 and FP32 hierarchies)."""
    macro = macro_by_name(name)
    meshes = [pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, level, coarsest_level=coarsest,
                       coarse_minres_max=30, **o) for o in (FUSED[fused], dict(fuse_coarse_levels=0))]
    H = MG.build_hierarchy(macro, level, coarsest=coarsest)
    st = _random_state(H, level, 21)
    for prec in (0, 1):
        outs = []
        for mesh in meshes:
            _load(mesh, H, level, st, precision=prec)
            mesh.level_op(level, "vcycle", precision=prec)
            outs.append(_read_up(mesh, H, level, precision=prec))
        tol = 1e-12 if prec == 0 else 1e-5
        assert rel_err(outs[0][0], outs[1][0]) < tol
        assert _p_err(H.levels[level], outs[0][1], outs[1][1]) < tol
