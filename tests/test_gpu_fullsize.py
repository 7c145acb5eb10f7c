"""Parity at the full size the bench times: the unit cube at level 9 (513^3
nodes, 5.35e8 free DoFs) with the default options, i.e. the kernels and
launch shapes of the bench (flags-first colour kernels, one plane per
colour block, backward velocity colour 0 fused with pressure colour 0, the
FP32 residual four nodes per thread, the refinement residual in fixed
point).  The oracle cannot assemble level 9; it computes sampled outputs
on windows of 33^3 lattice nodes (tests.helpers.LatticeWindow, checked
against the whole cube in test_oracle_windows.py), at two corners of the
cube, at one face and inside:
  * right-hand side (FP64): f at every interior node of a window; g up to
    the constant that the removal of its mean over the whole level adds
    (pure Dirichlet problem), and that mean is zero;
  * FP32 residual, restriction and prolongation: every output a window
    determines; one FP32 Uzawa step: the nodes at least 12 lattice steps
    from a held window face (one step per colour phase);
  * the refinement step of the FP32+IR mode (fixed-point update and FP64
    residual into the FP32 right-hand side): the iterate everywhere, the
    residual in the windows;
  * the bench's solve: FP32+IR to 1e-8 from zero in 8 cycles.
Tolerances as in test_gpu_parity.py: FP64 1e-12, FP32 steps 1e-5, the FP64
residual stored in FP32 1e-6, relative to the field's maximum over the
sampled nodes (the window's, for the random states of the kernel tests)."""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG
from tests.helpers import LatticeWindow, rel_err

pytestmark = pytest.mark.gpu

LEVEL = 9
DIM = (1 << LEVEL) + 1
WL = 5
# lattice origins: coordinate sums are multiples of 4 (the cube's colours)
# and even (the coarse lattice's nodes)
ORIGINS = [(0, 0, 0), (480, 480, 480), (240, 256, 16), (96, 300, 480)]
PHASES = 12
TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mesh(pkg):
    cube = W.unit_cube()
    m = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, LEVEL)
    yield m
    m.close()


@pytest.fixture(scope="module")
def windows():
    fine = [LatticeWindow(LEVEL, o, WL) for o in ORIGINS]
    coarse = [LatticeWindow(LEVEL - 1, tuple(c // 2 for c in o), WL - 1) for o in ORIGINS]
    return fine, coarse


def _state(torch, level, seed, fp32):
    """Seeded u, p, f, g of a level in lattice order (device, float64,
    rounded to FP32 values if fp32); u and f are zero on the cube's
    boundary (Dirichlet nodes)."""
    dim = (1 << level) + 1
    n = dim ** 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    out = []
    for shape in ((n, 3), (n,), (n, 3), (n,)):
        x = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64)
        out.append(x.float().double() if fp32 else x)
    idx = torch.arange(n, device="cuda")
    i, j, k = idx % dim, (idx // dim) % dim, idx // (dim * dim)
    e = dim - 1
    bnd = (i == 0) | (i == e) | (j == 0) | (j == e) | (k == 0) | (k == e)
    del idx, i, j, k
    out[0][bnd] = 0.0
    out[2][bnd] = 0.0
    return out


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


def test_level9_rhs_and_bench_solve(pkg, torch, mesh, windows):
    x = mesh.node_coords()
    mesh.set_rhs(W.manufactured_forcing(x), W.manufactured_velocity(x))
    del x
    F, G = _read(torch, mesh, LEVEL, "F", 0), _read(torch, mesh, LEVEL, "G", 0)
    assert abs(float(G.mean())) <= TOL64 * float(G.abs().max())
    outs = []
    for w in windows[0]:
        fn = W.manufactured_forcing(w.coords)
        ud = np.where(w.on_cube_boundary[:, None], W.manufactured_velocity(w.coords), 0.0)
        fu, g = w.L.rhs(fn, ud)
        outs.append((w, fu, g, *_at(torch, w, F, G)))
    del F, G
    # relative to the fields' maxima over the sampled nodes: the Dirichlet
    # lift makes them largest next to the boundary, which the corner windows
    # hold (inside the cube g is about 1e-9 of its maximum)
    sf = max(np.abs(fu).max() for _, fu, _, _, _ in outs)
    sg = max(np.abs(g[w.held_distance >= 1]).max() for w, _, g, _, _ in outs)
    for w, fu, g, gf, gg in outs:
        assert np.abs(gf[w.free] - fu.T).max() < TOL64 * sf
        rows = w.held_distance >= 1
        d = gg[rows] - g[rows]
        assert np.abs(d - d.mean()).max() < TOL64 * sg
    _, _, st = mesh.solve(tol=1e-8, max_cycles=50, mode=pkg.MODE_FP32_IR, want_solution=False)
    assert st.status == 0 and st.cycles == 8 and st.rel_residual <= 1e-8


def test_level9_fp32_kernels_sampled(pkg, torch, mesh, windows):
    u, p, f, g = _state(torch, LEVEL, 91, fp32=True)
    _write(torch, mesh, LEVEL, 1, U=u, P=p, F=f, G=g)
    mesh.level_op(LEVEL, "residual", precision=1)
    RU, RP = _read(torch, mesh, LEVEL, "RU", 1), _read(torch, mesh, LEVEL, "RP", 1)
    mesh.level_op(LEVEL, "restrict", precision=1)
    FC, GC = _read(torch, mesh, LEVEL - 1, "F", 1), _read(torch, mesh, LEVEL - 1, "G", 1)
    mesh.level_op(LEVEL, "uzawa_step", precision=1)
    U1, P1 = _read(torch, mesh, LEVEL, "U", 1), _read(torch, mesh, LEVEL, "P", 1)
    # prolongation of a seeded coarse correction onto the seeded fine state
    uc, pc = _state(torch, LEVEL - 1, 92, fp32=True)[:2]
    _write(torch, mesh, LEVEL, 1, U=u, P=p)
    _write(torch, mesh, LEVEL - 1, 1, U=uc, P=pc)
    mesh.level_op(LEVEL, "prolong_add", precision=1)
    U2, P2 = _read(torch, mesh, LEVEL, "U", 1), _read(torch, mesh, LEVEL, "P", 1)
    for w, cw in zip(*windows):
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
        assert rel_err(gu1[w.free][cf], wu.T[cf]) < TOL32
        assert rel_err(gp1[core], wp[core]) < TOL32
        # prolongation: every fine node of the window
        ucw, pcw = _at(torch, cw, uc, pc)
        free = ~w.on_cube_boundary
        assert rel_err(gu2[free], (uw + Pw @ ucw)[free]) < TOL32
        assert rel_err(gp2, pw + Pw @ pcw) < TOL32


def test_level9_refinement_sampled(pkg, torch, mesh, windows):
    x, q, f, g = _state(torch, LEVEL, 93, fp32=False)
    e, ep = _state(torch, LEVEL, 94, fp32=True)[:2]
    _write(torch, mesh, LEVEL, 0, U=x, P=q, F=f, G=g)
    _write(torch, mesh, LEVEL, 1, U=e, P=ep)
    mesh.level_op(LEVEL, "refine", precision=1)
    xu, xp = x + e, q + ep
    U, P = _read(torch, mesh, LEVEL, "U", 0), _read(torch, mesh, LEVEL, "P", 0)
    for got, want in ((U, xu), (P, xp)):
        bad = ((got - want).abs() > 1e-14 * float(want.abs().max())).reshape(len(want), -1).any(dim=1)
        where = torch.nonzero(bad).flatten()[:5].tolist()
        assert not bool(bad.any()), f"{int(bad.sum())} nodes differ, first {where}"
    RF, RG = _read(torch, mesh, LEVEL, "F", 1), _read(torch, mesh, LEVEL, "G", 1)
    for w in windows[0]:
        uw, pw, fw, gw = _at(torch, w, xu, xp, f, g)
        ru, rp = w.residual(uw, pw, fw, gw)
        grf, grg = _at(torch, w, RF, RG)
        rows = w.held_distance >= 1
        assert rel_err(grf[w.free], ru.T) < 1e-6
        assert rel_err(grg[rows], rp[rows]) < 1e-6
