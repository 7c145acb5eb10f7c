"""Parity at the full sizes the bench times, in its launch configuration
(default kernel options): the unit cube at level 9 (513^3 nodes, 5.35e8
free DoFs) and the obstacle channel at level 6 (1025 x 257 x 257 nodes,
2.6e8 free DoFs; coarsest level 1, coarse MINRES 5e-3 / 300), i.e.
flags-first colour kernels with one plane per colour block, backward
velocity colour 0 fused with pressure colour 0, the FP32 residual four
nodes per thread and the refinement residual in fixed point.  The oracle
cannot assemble these levels; it computes sampled outputs on windows of
33^3 lattice nodes (tests.helpers.LatticeWindow, checked against whole
domains in test_oracle_windows.py): on the cube at two corners, at one
face and inside; on the channel at an obstacle corner, along the edge two
obstacles share, on the inflow face and at the outflow face's corner.
  * right-hand side (FP64): f at every free node of a window; g up to the
    constant that the removal of its mean adds where a window or the domain
    is a pure Dirichlet problem, and on the cube that mean is zero;
  * FP32 residual, restriction and prolongation: every output a window
    determines; one FP32 Uzawa step: the nodes at least 12 lattice steps
    from a held window face (one step per colour phase);
  * the refinement step of the FP32+IR mode (fixed-point update and FP64
    residual into the FP32 right-hand side): the iterate everywhere, the
    residual in the windows;
  * the bench's solve: FP32+IR to 1e-8 from zero in its 8 (cube) or 9
    (channel) cycles.
Tolerances as in test_gpu_parity.py: FP64 1e-12, FP32 steps 1e-5, the FP64
residual stored in FP32 1e-6, relative to the field's maximum over the
sampled nodes (the window's, for the random states of the kernel tests)."""
import types

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG
from tests.helpers import LatticeWindow, rel_err

pytestmark = pytest.mark.gpu

WL = 5
PHASES = 12
TOL64 = 1e-12
TOL32 = 1e-5
# lattice origins: coordinate sums are multiples of 4 (the lattice's colours)
# and even (the coarse lattice's nodes)
CASES = {
    "cube9": dict(macro=W.unit_cube, level=9, opts={}, cycles=8,
                  origins=[(0, 0, 0), (480, 480, 480), (240, 256, 16), (96, 300, 480)]),
    "channel6": dict(macro=W.obstacle_channel, level=6, cycles=9,
                     opts=dict(coarsest_level=1, coarse_minres_max=300, coarse_minres_rtol=5e-3),
                     origins=[(48, 48, 112), (688, 112, 80), (0, 96, 96), (992, 0, 0)]),
}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    yield t
    t.cuda.empty_cache()   # the full-size states held tens of GB in torch's cache


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, pkg):
    c = CASES[request.param]
    macro = c["macro"]()
    level = c["level"]
    mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, level, **c["opts"])
    fine = [LatticeWindow(level, o, WL, domain=macro) for o in c["origins"]]
    coarse = [LatticeWindow(level - 1, tuple(v // 2 for v in o), WL - 1, domain=macro) for o in c["origins"]]
    yield types.SimpleNamespace(name=request.param, macro=macro, level=level, mesh=mesh, fine=fine, coarse=coarse,
                                cycles=c["cycles"])
    mesh.close()


def _masks(torch, macro, level):
    """Velocity Dirichlet nodes (walls, x = max without outflow, obstacle
    surfaces) and inactive nodes (in no remaining cell: inside an obstacle,
    or on a face or edge shared by obstacles only), on the device, in lattice
    order."""
    n_cell = 1 << level
    dims = macro.lattice_dims(level)
    idx = torch.arange(int(np.prod(dims)), device="cuda")
    g = (idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1]))
    del idx
    box = [c * n_cell for c in macro.cells]
    outflow = bool(np.any(macro.bc_flags == W.BC_OUTFLOW))
    dirichlet = (g[0] == 0) | (g[1] == 0) | (g[2] == 0) | (g[1] == box[1]) | (g[2] == box[2])
    if not outflow:
        dirichlet |= g[0] == box[0]
    for c in macro.removed:
        lo = [v * n_cell for v in c]
        dirichlet |= (g[0] >= lo[0]) & (g[0] <= lo[0] + n_cell) & (g[1] >= lo[1]) & (g[1] <= lo[1] + n_cell) & \
                     (g[2] >= lo[2]) & (g[2] <= lo[2] + n_cell)
    # a node is active when one of the (up to 8) cells whose closed box holds it is present
    present = torch.zeros([c + 2 for c in macro.cells], dtype=torch.bool, device="cuda")
    present[1:-1, 1:-1, 1:-1] = True
    for c in macro.removed:
        present[c[0] + 1, c[1] + 1, c[2] + 1] = False
    cand = [((a - 1).clamp(min=0) // n_cell + 1, torch.minimum(a // n_cell, torch.full_like(a, e)) + 1)
            for a, e in zip(g, macro.cells)]
    active = torch.zeros_like(dirichlet)
    for cx in cand[0]:
        for cy in cand[1]:
            for cz in cand[2]:
                active |= present[cx, cy, cz]
    return dirichlet, ~active


def _state(torch, case, seed, fp32):
    """Seeded u, p, f, g of the finest level in lattice order (device,
    float64, rounded to FP32 values if fp32); u and f are zero on Dirichlet
    nodes, all four at inactive nodes."""
    n = case.mesh.num_nodes(case.level)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    out = []
    for shape in ((n, 3), (n,), (n, 3), (n,)):
        x = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64)
        out.append(x.float().double() if fp32 else x)
    dirichlet, inactive = _masks(torch, case.macro, case.level)
    out[0][dirichlet] = 0.0
    out[2][dirichlet] = 0.0
    out[1][inactive] = 0.0
    out[3][inactive] = 0.0
    return out


def _coarse_state(torch, case, seed):
    """Seeded FP32-valued u, p of the next coarser level, zero where it has no unknowns."""
    level = case.level - 1
    n = case.mesh.num_nodes(level)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    u = torch.randn((n, 3), generator=gen, device="cuda", dtype=torch.float64).float().double()
    p = torch.randn((n,), generator=gen, device="cuda", dtype=torch.float64).float().double()
    dirichlet, inactive = _masks(torch, case.macro, level)
    u[dirichlet] = 0.0
    p[inactive] = 0.0
    return u, p


def _at(torch, w, *fields):
    idx = torch.from_numpy(w.index).cuda()
    return [x[idx].cpu().numpy() for x in fields]


def _read(torch, mesh, level, field, precision):
    n = mesh.num_nodes(level)
    out = torch.empty((n, 3) if field in ("U", "F", "RU") else (n,), dtype=torch.float64, device="cuda")
    mesh.level_field(level, field, precision, out=out)
    return out


def _write(torch, mesh, level, precision, **fields):
    # the mesh's own stream does not wait on torch's: the inputs must be complete
    torch.cuda.synchronize()
    for name, v in fields.items():
        mesh.level_field(level, name, precision, v)


def _rhs_inputs(case):
    """The nodal body force and Dirichlet data of the parity check: the
    manufactured solution on the cube, a seeded N(0,1) force and the inflow
    profile on the channel."""
    x = case.mesh.node_coords()
    if case.name.startswith("cube"):
        return (lambda c, idx: W.manufactured_forcing(c)), W.manufactured_forcing(x), W.manufactured_velocity, \
            W.manufactured_velocity(x)
    fn = W.random_body_force(x.shape[0], seed=4)
    return (lambda c, idx: fn[idx]), fn, W.channel_inflow, W.channel_inflow(x)


def test_rhs_and_bench_solve(pkg, torch, case):
    mesh, level = case.mesh, case.level
    f_of, fn, ud_of, ud = _rhs_inputs(case)
    mesh.set_rhs(fn, ud)
    del fn, ud
    F, G = _read(torch, mesh, level, "F", 0), _read(torch, mesh, level, "G", 0)
    if case.name.startswith("cube"):
        assert abs(float(G.mean())) <= TOL64 * float(G.abs().max())
    outs = []
    for w in case.fine:
        udw = np.where(w.dirichlet[:, None], ud_of(w.coords), 0.0)
        fu, g = w.L.rhs(f_of(w.coords, w.index), udw)
        outs.append((w, fu, g, *_at(torch, w, F, G)))
    del F, G
    # relative to the fields' maxima over the sampled nodes: the Dirichlet
    # lift makes them largest next to the boundary, which windows hold
    # (inside the cube g is about 1e-9 of its maximum)
    sf = max(np.abs(fu).max() for _, fu, _, _, _ in outs)
    sg = max(np.abs(g[w.held_distance >= 1]).max() for w, _, g, _, _ in outs)
    for w, fu, g, gf, gg in outs:
        assert np.abs(gf[w.free] - fu.T).max() < TOL64 * sf
        rows = w.held_distance >= 1
        d = gg[rows] - g[rows]
        assert np.abs(d - d.mean()).max() < TOL64 * sg
    # the bench's solve
    if not case.name.startswith("cube"):
        mesh.set_rhs(None, W.channel_inflow(mesh.node_coords()))
    _, _, st = mesh.solve(tol=1e-8, max_cycles=60, mode=pkg.MODE_FP32_IR, want_solution=False)
    assert st.status == 0 and st.cycles == case.cycles and st.rel_residual <= 1e-8


def test_fp32_kernels_sampled(pkg, torch, case):
    mesh, level = case.mesh, case.level
    u, p, f, g = _state(torch, case, 91, fp32=True)
    _write(torch, mesh, level, 1, U=u, P=p, F=f, G=g)
    mesh.level_op(level, "residual", precision=1)
    RU, RP = _read(torch, mesh, level, "RU", 1), _read(torch, mesh, level, "RP", 1)
    mesh.level_op(level, "restrict", precision=1)
    FC, GC = _read(torch, mesh, level - 1, "F", 1), _read(torch, mesh, level - 1, "G", 1)
    mesh.level_op(level, "uzawa_step", precision=1)
    U1, P1 = _read(torch, mesh, level, "U", 1), _read(torch, mesh, level, "P", 1)
    # prolongation of a seeded coarse correction onto the seeded fine state
    uc, pc = _coarse_state(torch, case, 92)
    _write(torch, mesh, level, 1, U=u, P=p)
    _write(torch, mesh, level - 1, 1, U=uc, P=pc)
    mesh.level_op(level, "prolong_add", precision=1)
    U2, P2 = _read(torch, mesh, level, "U", 1), _read(torch, mesh, level, "P", 1)
    for w, cw in zip(case.fine, case.coarse):
        uw, pw, fw, gw = _at(torch, w, u, p, f, g)
        gru, grp, gu1, gp1, gu2, gp2 = _at(torch, w, RU, RP, U1, P1, U2, P2)
        rows = w.held_distance >= 1
        ru, rp = w.residual(uw, pw, fw, gw)
        assert rel_err(gru[w.free], ru.T) < TOL32
        assert rel_err(grp[rows], rp[rows]) < TOL32
        # restriction: the coarse nodes inside the window
        Pw = MG.prolongation(w.L, cw.L)
        r_full = np.zeros((len(w.index), 3))
        r_full[w.free] = ru.T
        gfc, ggc = _at(torch, cw, FC, GC)
        assert rel_err(gfc[cw.free], (Pw.T @ r_full)[cw.free]) < TOL32
        assert rel_err(ggc[cw.free], (Pw.T @ np.where(rows, rp, 0.0))[cw.free]) < TOL32
        # one Uzawa step: the core of the window
        wu, wp = w.uzawa_step(uw, pw, fw, gw)
        core = w.held_distance >= PHASES
        cf = core[w.free]
        assert cf.sum() > 0
        assert rel_err(gu1[w.free][cf], wu.T[cf]) < TOL32
        assert rel_err(gp1[core], wp[core]) < TOL32
        # prolongation: every fine node of the window
        ucw, pcw = _at(torch, cw, uc, pc)
        free = ~w.dirichlet
        assert rel_err(gu2[free], (uw + Pw @ ucw)[free]) < TOL32
        assert rel_err(gp2, pw + Pw @ pcw) < TOL32


def test_refinement_sampled(pkg, torch, case):
    mesh, level = case.mesh, case.level
    x, q, f, g = _state(torch, case, 93, fp32=False)
    e, ep = _state(torch, case, 94, fp32=True)[:2]
    _write(torch, mesh, level, 0, U=x, P=q, F=f, G=g)
    _write(torch, mesh, level, 1, U=e, P=ep)
    mesh.level_op(level, "refine", precision=1)
    xu, xp = x + e, q + ep
    U, P = _read(torch, mesh, level, "U", 0), _read(torch, mesh, level, "P", 0)
    for got, want in ((U, xu), (P, xp)):
        bad = ((got - want).abs() > 1e-14 * float(want.abs().max())).reshape(len(want), -1).any(dim=1)
        where = torch.nonzero(bad).flatten()[:5].tolist()
        assert not bool(bad.any()), f"{int(bad.sum())} nodes differ, first {where}"
    RF, RG = _read(torch, mesh, level, "F", 1), _read(torch, mesh, level, "G", 1)
    for w in case.fine:
        uw, pw, fw, gw = _at(torch, w, xu, xp, f, g)
        ru, rp = w.residual(uw, pw, fw, gw)
        grf, grg = _at(torch, w, RF, RG)
        rows = w.held_distance >= 1
        assert rel_err(grf[w.free], ru.T) < 1e-6
        assert rel_err(grg[rows], rp[rows]) < 1e-6
