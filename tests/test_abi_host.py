"""C ABI checks that need no GPU: the library builds, loads and exports every
function declared in include/hhg_stokes.h; the host-side lattice
classification agrees with the oracle's refined mesh; bad macro meshes are
rejected with error codes."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import mesh as M
from tests.helpers import macro_by_name

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_02134_gb300 as p
    return p


def test_exports_every_declared_symbol(pkg):
    header = open(os.path.join(ROOT, "include", "hhg_stokes.h")).read()
    declared = set(re.findall(r"^\s*(?:void|int|const char\*)\s+(hhg_\w+)\s*\(", header, re.M))
    assert len(declared) >= 20
    lib = pkg.load_library()
    for name in sorted(declared):
        assert hasattr(lib, name), name


@pytest.mark.parametrize("name,levels", [("cube", (0, 1, 2, 3)), ("channel", (0, 1, 2)), ("partial", (1, 2, 3))])
def test_classification_matches_oracle(pkg, name, levels):
    macro = macro_by_name(name)
    for lev in levels:
        dims, fl = pkg.lattice_classify(macro.vertices, macro.tets, macro.bc_flags, lev)
        r = M.refine(macro.vertices, macro.tets, macro.bc_flags, lev)
        lat = r.ijk[:, 0] + dims[0] * (r.ijk[:, 1] + dims[1] * r.ijk[:, 2])
        act = np.zeros(len(fl), bool)
        act[lat] = True
        vf = np.zeros(len(fl), bool)
        vf[lat[r.free_velocity]] = True
        cnt = np.bincount(r.tets.ravel(), minlength=r.n_nodes)
        irr = np.zeros(len(fl), bool)
        irr[lat[cnt < 24]] = True
        out = np.zeros(len(fl), bool)
        out[lat[r.on_outflow]] = True
        assert np.array_equal(act, (fl & pkg.NODE_ACTIVE) > 0)
        assert np.array_equal(vf, (fl & pkg.NODE_VFREE) > 0)
        assert np.array_equal(irr, (fl & pkg.NODE_IRREG) > 0)
        assert np.array_equal(out, (fl & pkg.NODE_OUTFLOW) > 0)


def test_rejects_bad_meshes(pkg):
    cube = W.unit_cube()
    # vertex order not along a lattice path
    T = cube.tets.copy()
    T[0] = T[0][[0, 2, 1, 3]]
    with pytest.raises(pkg.HHGError) as e:
        pkg.lattice_classify(cube.vertices, T, cube.bc_flags, 1)
    assert e.value.code == -2
    # duplicate tetrahedron
    T = np.concatenate([cube.tets, cube.tets[:1]])
    with pytest.raises(pkg.HHGError) as e:
        pkg.lattice_classify(cube.vertices, T, None, 1)
    assert e.value.code == -2
    # vertex id out of range
    T = cube.tets.copy()
    T[0, 0] = 99
    with pytest.raises(pkg.HHGError) as e:
        pkg.lattice_classify(cube.vertices, T, None, 1)
    assert e.value.code == -1
    # vertex off the lattice
    V = cube.vertices.copy()
    V[7] += 0.3
    with pytest.raises(pkg.HHGError) as e:
        pkg.lattice_classify(V, cube.tets, None, 1)
    assert e.value.code == -2


def test_create_mesh_without_gpu_fails_cleanly(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cube = W.unit_cube()
    with pytest.raises(pkg.HHGError) as e:
        pkg.Mesh(cube.vertices, cube.tets, cube.bc_flags, 2)
    assert e.value.code == -6
