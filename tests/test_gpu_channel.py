"""The obstacle channel (16 x 4 x 4 unit cubes, 6 seeded obstacle cubes,
parabolic inflow, do-nothing outflow; the synthetic stand-in for the sphere
bed of Sec. 6) at level 4, 4.0e6 free DoFs, against the oracle.

The coarse MINRES is tolerance-driven (relative 5e-3, at most 300
iterations, Sec. 3.7), so per-cycle rounding differences pass through a long
Krylov recurrence: FP64 solutions agree to 1e-9 and the residual histories
to 1e-6.  FP32+IR reaches 1e-8 with an error against the oracle's solution
(1e-10) within 10x of the error the oracle's own FP64 iterate has at 1e-8.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG
from tests.helpers import lattice_index, rel_err

pytestmark = pytest.mark.gpu

LEVEL, COARSEST, MX, RTOL = 4, 1, 300, 5e-3


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


@pytest.fixture(scope="module")
def oracle():
    ch = W.obstacle_channel()
    H = MG.build_hierarchy(ch, LEVEL, coarsest=COARSEST, opt=MG.Options(coarse_minres_max=MX, coarse_minres_rtol=RTOL))
    L = H.levels[LEVEL]
    x = L.mesh.xyz
    ud = W.channel_inflow(x)
    f, g = L.rhs(np.zeros_like(x), ud)
    res = MG.solve(H, f, g, tol=1e-10, max_cycles=40, keep_iterates=True)
    return H, ud, res


def test_channel_level4_fp64_and_fp32ir_match_oracle(pkg, oracle):
    H, ud, ref = oracle
    L = H.levels[LEVEL]
    ch = W.obstacle_channel()
    mesh = pkg.Mesh(ch.vertices, ch.tets, ch.bc_flags, LEVEL, coarsest_level=COARSEST, coarse_minres_max=MX,
                    coarse_minres_rtol=RTOL)
    x = mesh.node_coords()
    lat = lattice_index(L, mesh.dims())
    mesh.set_rhs(None, W.channel_inflow(x))
    u, p, st = mesh.solve(tol=1e-10, max_cycles=40, mode=pkg.MODE_FP64)
    assert st.status == 0 and st.cycles == ref.cycles
    np.testing.assert_allclose(st.history, ref.history, rtol=1e-6, atol=1e-13)
    u_ref = L.scatter(ref.u, ud)
    assert rel_err(u[lat], u_ref) < 1e-9 and rel_err(p[lat], ref.p) < 1e-9
    # FP32+IR to 1e-8, against the oracle's own iterate at the same tolerance
    k8 = next(c for c, h in enumerate(ref.history) if h <= 1e-8)
    u8, p8 = ref.iterates[k8 - 1]
    eu64, ep64 = rel_err(L.scatter(u8, ud), u_ref), rel_err(p8, ref.p)
    mesh.set_rhs(None, W.channel_inflow(x))
    u32, p32, s32 = mesh.solve(tol=1e-8, max_cycles=40, mode=pkg.MODE_FP32_IR)
    assert s32.status == 0 and s32.rel_residual <= 1e-8
    eu, ep = rel_err(u32[lat], u_ref), rel_err(p32[lat], ref.p)
    print("channel level 4 FP32+IR cycles", s32.cycles, "err u", eu, "vs", eu64, "err p", ep, "vs", ep64)
    assert eu <= 10 * eu64 + 1e-9 and ep <= 10 * ep64 + 1e-7
    mesh.close()
