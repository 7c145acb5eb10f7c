"""C ABI checks that need no GPU: the library builds, loads and exports every
function declared in include/hhg_stokes.h; the host-side lattice
classification agrees with the oracle's refined mesh; the operator the
kernels apply, assembled on the host from the same stencil classes and
closed-form rows, equals the oracle's assembled K entry by entry; bad macro
meshes are rejected with error codes."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import mesh as M
from oracle import stokes as S
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


@pytest.mark.parametrize("name,levels", [("cube", (0, 1, 2, 3)), ("channel", (0, 1, 2)), ("partial", (1, 2, 3)),
                                         ("sheared", (1, 2, 3)), ("slip_channel", (0, 1, 2)),
                                         ("slip_cube", (1, 2, 3)), ("sheared_slip", (1, 2)),
                                         ("slip_obstacle", (1, 2))])
def test_classification_matches_oracle(pkg, name, levels):
    macro = macro_by_name(name)
    affine = macro.basis is not None
    for lev in levels:
        dims, fl = pkg.lattice_classify(macro.vertices, macro.tets, macro.bc_flags, lev)
        r = M.refine(macro.vertices, macro.tets, macro.bc_flags, lev, basis=macro.basis)
        if (np.asarray(macro.bc_flags) == 3).any():
            S.build_level(r)  # free-slip nodes without a normal become Dirichlet nodes (in place)
        lat = r.ijk[:, 0] + dims[0] * (r.ijk[:, 1] + dims[1] * r.ijk[:, 2])
        act = np.zeros(len(fl), bool)
        act[lat] = True
        vf = np.zeros(len(fl), bool)
        vf[lat[r.free_velocity]] = True
        cnt = np.bincount(r.tets.ravel(), minlength=r.n_nodes)
        irr = np.zeros(len(fl), bool)
        irr[lat[(cnt < 24) | affine]] = True   # affine lattices: every active node takes class rows
        out = np.zeros(len(fl), bool)
        out[lat[r.on_outflow]] = True
        slip = np.zeros(len(fl), bool)
        slip[lat[r.on_slip & r.free_velocity]] = True
        assert np.array_equal(slip, (fl & pkg.NODE_SLIP) > 0)
        assert np.all((fl[slip] & pkg.NODE_IRREG) > 0)
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


def _struct_fields(header, name):
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), header, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"^\s*(double|int32_t|int64_t)\s+(\w+)(\[\d+\])?\s*;", body, re.M)


def test_binding_mirrors_header(pkg, tmp_path):
    """The Python binding's op codes and ctypes structs match the C header:
    names, order, types, and (compiled with the host C compiler) offsets and
    sizes."""
    import ctypes
    import shutil
    import subprocess
    header = open(os.path.join(ROOT, "include", "hhg_stokes.h")).read()
    ops = {m[0].lower(): int(m[1]) for m in re.findall(r"#define HHG_OP_(\w+)\s+(\d+)", header)}
    assert ops == pkg.OP
    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64}
    for cname, py in (("hhg_options", pkg.Options), ("hhg_stats", pkg._Stats)):
        fields = _struct_fields(header, cname)
        assert [f[1] for f in fields] == [f[0] for f in py._fields_], cname
        for (ty, nm, arr), (pn, pt) in zip(fields, py._fields_):
            want = ctype[ty] * int(arr[1:-1]) if arr else ctype[ty]
            assert ctypes.sizeof(pt) == ctypes.sizeof(want) and getattr(pt, "_type_", pt) == getattr(want, "_type_", want), nm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hhg_stokes.h"', "int main(void) {"]
    for cname in ("hhg_options", "hhg_stats"):
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for _, nm, _ in _struct_fields(header, cname):
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, nm, cname, nm))
    lines += ["return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if l)
    for cname, py in (("hhg_options", pkg.Options), ("hhg_stats", pkg._Stats)):
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for pn, _ in py._fields_:
            assert int(got["%s.%s" % (cname, pn)]) == getattr(py, pn).offset, (cname, pn)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("name,level", [("cube", 2), ("channel", 1), ("partial", 2), ("sheared", 2),
                                        ("slip_channel", 1), ("slip_cube", 2), ("sheared_slip", 2),
                                        ("slip_obstacle", 2)])
def test_host_operator_equals_oracle_matrix(pkg, name, level, form):
    """K of a level from the stencil classes (boundary rows), the closed-form
    rows (full-star nodes) and the scale factors the kernels use, against the
    oracle's K assembled from element integrals (Sec. 2.1 forms; free slip
    constrained as in Sec. 6.1), after matching the unknowns by their nodes:
    each of the four blocks (A, B^T, B, -C) to 1e-12 of its largest entry;
    and the lumped pressure mass of the class tables against the oracle's."""
    import scipy.sparse as sp
    macro = macro_by_name(name)
    kptr, kcol, kval, vnode, pnode, pmass = pkg.assemble_operator_host(macro.vertices, macro.tets, macro.bc_flags,
                                                                       level, operator_form=form)
    L = S.build_from_macro(macro, level, form="D" if form else "laplace")
    dims = macro.lattice_dims(level)
    lat = L.mesh.ijk[:, 0] + dims[0] * (L.mesh.ijk[:, 1] + dims[1] * L.mesh.ijk[:, 2])
    node_of = np.full(int(np.prod(dims)), -1)
    node_of[lat] = np.arange(len(lat))
    free_pos = np.full(L.n_p, -1)
    free_pos[L.free] = np.arange(L.n_u)
    nv, nu_ = len(vnode), L.n_u
    assert nv == nu_ and len(pnode) == L.n_p
    q = free_pos[node_of[vnode]]
    assert np.all(q >= 0) and len(np.unique(q)) == nv
    perm = np.concatenate([d * nu_ + q for d in range(3)] + [3 * nu_ + node_of[pnode]])
    n = len(perm)
    Kh = sp.csr_matrix((kval, kcol, kptr), shape=(n, n))
    Ko = S.full_matrix(L).tocsr()[perm][:, perm]
    for rs in (slice(0, 3 * nv), slice(3 * nv, n)):
        for cs in (slice(0, 3 * nv), slice(3 * nv, n)):
            ref = Ko[rs, cs]
            diff = abs(Kh[rs, cs] - ref).max()
            assert diff <= 1e-12 * abs(ref).max(), (name, form, rs, cs, diff, abs(ref).max())
    np.testing.assert_allclose(pmass, L.m[node_of[pnode]], rtol=1e-13)
