"""The allocation-free coarse-grid solve (hhg_coarse_solve_noalloc) against
the allocating path (level fields + hhg_level_op(COARSE_SOLVE)).

Callers that may not allocate device memory after set-up (fixed arenas,
framework-owned pools, latency-bound loops) use the allocation-free entry
point; it must give the same corrected iterate as the regular coarse solve.
Two calls in a row, with different data, check that the shared scratch array
carries nothing from one call into the next, and that neither call allocates:
the mesh's allocation counter (every cudaMalloc / cudaMallocHost it makes,
temporaries included) and the device's free memory are unchanged across it.
A call rejected for size writes nothing.  This file is collected last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


def _data(mesh, level, seed):
    n = mesh.num_nodes(level)
    flags = mesh.node_flags(level)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, 3))
    g = rng.standard_normal(n)
    act = (flags & 1) > 0
    if not (flags & 16).any():          # no outflow: make g consistent with K's null vector
        g[act] -= g[act].mean()
    return f, g, rng.standard_normal((n, 3)), rng.standard_normal(n)


def _reference(mesh, level, f, g, u, p):
    mesh.level_field(level, "F", 0, f)
    mesh.level_field(level, "G", 0, g)
    mesh.level_field(level, "U", 0, u)
    mesh.level_field(level, "P", 0, p)
    mesh.level_op(level, "coarse_solve")
    return mesh.level_field(level, "U"), mesh.level_field(level, "P")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name,finest,coarsest,mx", [("cube", 3, 2, 5), ("channel", 2, 1, 40)])
def test_noalloc_matches_coarse_solve(pkg, name, finest, coarsest, mx):
    macro = W.unit_cube() if name == "cube" else W.obstacle_channel()
    mesh = pkg.Mesh(macro.vertices, macro.tets, macro.bc_flags, finest, coarsest_level=coarsest,
                    coarse_minres_max=mx)
    flags = mesh.node_flags(coarsest)
    vf, act = (flags & 2) > 0, (flags & 1) > 0
    import torch
    for call, seed in enumerate((1, 2)):
        f, g, u, p = _data(mesh, coarsest, seed)
        ur, pr = _reference(mesh, coarsest, f, g, u, p)
        u2, p2 = u.copy(), p.copy()
        torch.cuda.synchronize()
        allocs, free0 = mesh.allocations(), torch.cuda.mem_get_info()[0]
        mesh.coarse_solve_noalloc(f, g, u2, p2)
        torch.cuda.synchronize()
        assert mesh.allocations() == allocs, call
        assert torch.cuda.mem_get_info()[0] == free0, call
        assert _rel(u2[vf], ur[vf]) <= 1e-12, call
        assert _rel(p2[act], pr[act]) <= 1e-12, call
        assert np.all(u2[~vf] == 0) and np.all(p2[~act] == 0)
    mesh.close()


def test_noalloc_rejects_large_coarse_level(pkg):
    cube = W.unit_cube()
    mesh = pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 5, coarsest_level=5)
    n = mesh.num_nodes(5)
    f, g, u, p = _data(mesh, 5, 3)
    for name, val in (("F", f), ("G", g), ("U", u), ("P", p)):
        mesh.level_field(5, name, 0, val)
    before = {name: mesh.level_field(5, name) for name in ("F", "G", "U", "P")}
    u_in, p_in = np.ones((n, 3)), np.ones(n)
    allocs = mesh.allocations()
    with pytest.raises(pkg.HHGError) as e:
        mesh.coarse_solve_noalloc(np.zeros((n, 3)), np.zeros(n), u_in, p_in)
    assert e.value.code == -1 and "scratch" in str(e.value)
    assert mesh.allocations() == allocs
    # nothing written: neither the caller's arrays nor the mesh's fields
    assert np.all(u_in == 1.0) and np.all(p_in == 1.0)
    for name, val in before.items():
        assert np.array_equal(mesh.level_field(5, name), val), name
    mesh.close()
