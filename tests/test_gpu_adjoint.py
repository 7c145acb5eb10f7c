"""Adjoint gradient on the GPU (obstacle channel, level 5).

J_psi(u) = sum_i psi_i w_i . u_i is the outflow flux weighted by
psi = y z / 16 (the unweighted flux does not depend on the body force, see
the oracle pins).  Checked against the oracle's direct adjoint gradient on a
small level, and against central finite differences at level 5 on 32 seeded
directions with step 1e-6: each perturbed solve starts from the base
solution (solved to 1e-12) and is iterated to 1e-9 relative to its own
initial residual (at least 1e-8 must be reached), so the finite difference
carries only that algebraic error (J is affine in f).  The differences are taken on the f-dependent
part of J (zero Dirichlet data): the inflow adds a constant that would
only cancel in FP64.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, multigrid as MG
from tests.helpers import lattice_index, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


def test_autograd_matches_oracle_gradient(pkg):
    torch = pytest.importorskip("torch")
    from paper_1511_02134_gb300.autograd import stokes_solve
    ch = W.obstacle_channel()
    mesh = pkg.Mesh(ch.vertices, ch.tets, ch.bc_flags, 2, coarsest_level=1, coarse_minres_max=300)
    x = mesh.node_coords()
    Wt = torch.from_numpy(mesh.outflow_weights() * W.outflow_flux_weight(x)[:, None]).cuda()
    ud = torch.from_numpy(W.channel_inflow(x)).cuda()
    f = torch.from_numpy(W.random_body_force(len(x), seed=1)).cuda().requires_grad_(True)
    u, p = stokes_solve(f, mesh, ud, tol=1e-12, max_cycles=80)
    J = (Wt * u).sum()
    J.backward()
    L = MG.build_hierarchy(ch, 2, coarsest=1).levels[2]
    lat = lattice_index(L, mesh.dims())
    ref = adjoint.gradient_direct(L, W.outflow_flux_weight(L.mesh.xyz))
    assert rel_err(f.grad.cpu().numpy()[lat], ref) < 1e-9
    # the forward value matches the oracle's direct solution
    jref = adjoint.functional_direct(L, W.random_body_force(len(x), seed=1)[lat], W.channel_inflow(x)[lat],
                                     W.outflow_flux_weight(L.mesh.xyz))
    assert float(J.detach()) == pytest.approx(jref, rel=1e-9)


@pytest.mark.slow
def test_gradient_vs_finite_differences_level5(pkg):
    ch = W.obstacle_channel()
    mesh = pkg.Mesh(ch.vertices, ch.tets, ch.bc_flags, 5, coarsest_level=1, coarse_minres_max=300)
    x = mesh.node_coords()
    n = len(x)
    Wj = mesh.outflow_weights() * W.outflow_flux_weight(x)[:, None]
    f0 = W.random_body_force(n, seed=1)
    # J is affine in f; the Dirichlet inflow only adds an f-independent
    # constant (about 7) that would cancel in every difference, so the
    # differences are taken on the f-dependent part (zero Dirichlet data),
    # which has the same gradient
    mesh.set_rhs(f0, None)
    u0, p0, st = mesh.solve(tol=1e-12, max_cycles=80)
    assert st.status == 0
    grad, st = mesh.adjoint_gradient(ju=Wj, tol=1e-12, max_cycles=80)
    assert st.status == 0
    eps = 1e-6
    dirs = W.random_directions(n, count=32, seed=2)
    worst = 0.0
    for d in dirs:
        js = []
        for sgn in (1.0, -1.0):
            mesh.set_rhs(f0 + sgn * eps * d, None)
            mesh.set_initial(u0, p0)
            u, _, s = mesh.solve(tol=1e-9, max_cycles=40)
            assert s.rel_residual <= 1e-8
            js.append(float(np.sum(Wj * u)))
        fd = (js[0] - js[1]) / (2 * eps)
        an = float(np.sum(grad * d))
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst <= 1e-6, worst
