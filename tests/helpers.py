"""Test helpers: mapping between the oracle's node numbering and the lattice
order used by the C ABI (nodes are matched by their lattice coordinates)."""
import numpy as np

import workloads as W


def lattice_index(L, dims):
    ijk = L.mesh.ijk
    return ijk[:, 0] + dims[0] * (ijk[:, 1] + dims[1] * ijk[:, 2])


def u_to_lattice(L, dims, u):
    """(3, n_u) free-node velocity -> (n_lat, 3) with zeros elsewhere."""
    out = np.zeros((int(np.prod(dims)), 3))
    lat = lattice_index(L, dims)
    out[lat[L.free]] = np.asarray(u).T
    return out


def p_to_lattice(L, dims, p):
    out = np.zeros(int(np.prod(dims)))
    out[lattice_index(L, dims)] = p
    return out


def u_from_lattice(L, dims, arr):
    lat = lattice_index(L, dims)
    return np.asarray(arr)[lat[L.free]].T.copy()


def p_from_lattice(L, dims, arr):
    return np.asarray(arr)[lattice_index(L, dims)].copy()


def nodal_to_lattice(L, dims, arr_nodes):
    """(n_oracle_nodes, k) -> (n_lat, k)."""
    arr_nodes = np.asarray(arr_nodes)
    out = np.zeros((int(np.prod(dims)),) + arr_nodes.shape[1:])
    out[lattice_index(L, dims)] = arr_nodes
    return out


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


def macro_by_name(name):
    if name == "cube":
        return W.unit_cube()
    if name == "channel":
        return W.obstacle_channel()
    if name == "sheared":
        return W.sheared_cube()
    if name == "slip_channel":
        return W.slip_channel()
    if name == "slip_cube":
        return W.slip_cube()
    if name == "sheared_slip":
        return W.sheared_slip_cube()
    if name == "slip_obstacle":
        # one free-slip obstacle cube inside a box of Dirichlet walls
        return W.box_of_cubes(3, 3, 3, removed=((1, 1, 1),), slip_obstacles=True)
    if name == "partial":
        # two unit cubes with two Kuhn tetrahedra removed and one listed along
        # its reversed path: partially filled macro cells, irregular rows inside
        m = W.box_of_cubes(2, 1, 1)
        keep = [t for t in range(len(m.tets)) if t not in (1, 4)]
        T = m.tets[keep].copy()
        T[3] = T[3][::-1]
        m.tets = T
        m.bc_flags = np.zeros_like(T, dtype=np.uint8)
        return m
    raise KeyError(name)


class LatticeWindow:
    """A block of (2^wl + 1)^3 nodes of the Kuhn lattice at `level` of a box
    of unit cubes (`domain`, a workloads.box_of_cubes mesh, default the unit
    cube: obstacle cells removed, no-slip walls, optionally do-nothing
    outflow on x = max), from lattice coordinates `origin`, assembled by
    the oracle.  With the origin on multiples of 2^(wl-1) the block is
    2 x 2 x 2 sub-cells, each inside one unit cube, and sub-cells inside an
    obstacle are left out; otherwise it is one cell and must meet no
    obstacle.  The oracle refines this small box of cubes (the same Kuhn
    lattice, which is invariant under lattice translations) and scales and
    moves it onto the block.  Every row of a
    node off the block's faces is the row of the whole domain there, so the
    oracle can produce sampled outputs of levels it cannot assemble.

    The block's faces are Dirichlet faces of its oracle level, except an
    outflow face of the domain.  Where they lie on the domain's walls or
    obstacles they are Dirichlet faces of the domain too; elsewhere (the
    "held" faces) they stand for nodes whose rows reach outside the block and
    keep the values they are given."""

    def __init__(self, level, origin, wl, domain=None):
        import itertools

        from oracle import mesh as OM
        from oracle import stokes as S
        dom = W.unit_cube() if domain is None else domain
        if np.any(dom.bc_flags == W.BC_SLIP):
            raise NotImplementedError("windows of free-slip domains")
        out_faces = dom.bc_flags == W.BC_OUTFLOW
        has_outflow = bool(out_faces.any())
        n_cell, width = 1 << level, 1 << wl
        origin = np.asarray(origin, np.int64)
        box = np.asarray(dom.cells, np.int64) * n_cell
        end = origin + width
        assert np.all(origin >= 0) and np.all(end <= box)
        rset = set(tuple(c) for c in dom.removed)
        if np.all(origin % (width // 2) == 0) and width // 2 <= n_cell:
            k = 2   # 2 x 2 x 2 sub-cells, each inside one unit cube
        else:
            k = 1   # one cell: the block must meet no obstacle
            lo, hi = origin // n_cell, (end - 1) // n_cell
            assert not any(c in rset for c in itertools.product(*(range(a, b + 1) for a, b in zip(lo, hi))))
        sub = width // k
        removed = [c for c in itertools.product(range(k), repeat=3)
                   if tuple(int(v) for v in (origin + sub * np.asarray(c)) // n_cell) in rset]
        macro = W.box_of_cubes(k, k, k, removed=removed, outflow_x_max=has_outflow and end[0] == box[0])
        m = OM.refine(macro.vertices, macro.tets, macro.bc_flags, wl - (k - 1))
        m.ijk = m.key.copy()   # local lattice coordinates 0 .. 2^wl
        scale = sub / float(n_cell)
        m.xyz = m.xyz * scale + origin / float(n_cell)
        m.h = m.h * scale
        self.level, self.wl, self.origin = level, wl, origin
        self.L = S.build_level(m)
        self.ijk = m.ijk
        self.glob = m.ijk + origin
        dims = box + 1
        self.index = self.glob[:, 0] + dims[0] * (self.glob[:, 1] + dims[1] * self.glob[:, 2])
        self.coords = self.glob / float(n_cell)
        # velocity Dirichlet nodes of the domain: walls (and x = max without
        # outflow) and the closed boxes of the obstacle cells
        g = self.glob
        wall = (g[:, 0] == 0) | (g[:, 1] == 0) | (g[:, 2] == 0) | (g[:, 1] == box[1]) | (g[:, 2] == box[2])
        if not has_outflow:
            wall |= g[:, 0] == box[0]
        for c in rset:
            lo = np.asarray(c) * n_cell
            wall |= np.all((g >= lo) & (g <= lo + n_cell), axis=1)
        self.dirichlet = wall
        held = np.full(len(g), np.iinfo(np.int64).max)
        for a in range(3):
            if origin[a] > 0:
                held = np.minimum(held, self.ijk[:, a])
            if end[a] < box[a]:
                held = np.minimum(held, width - self.ijk[:, a])
        self.held_distance = held

    @property
    def free(self):
        return self.L.free

    def lift(self, u, f, g):
        """The window's right-hand side with its boundary nodes' velocities
        u (n, 3) moved into it: f at the free nodes (3, n_free) and g (n,)."""
        L, ops = self.L, self.L.ops
        fr, bd = L.free, L.dir
        fl = np.stack([f[fr, d] - ops.A[fr][:, bd] @ u[bd, d] for d in range(3)])
        gl = g - sum(ops.B[d][:, bd] @ u[bd, d] for d in range(3))
        return fl, gl

    def residual(self, u, p, f, g):
        """(f, g) - K (u, p) of the window from nodal u (n, 3), p, f (n, 3), g:
        ru (3, n_free), rp (n,); rows of the boundary nodes are incomplete."""
        fl, gl = self.lift(u, f, g)
        return self.L.residual(u[self.L.free].T, p, fl, gl)

    def uzawa_step(self, u, p, f, g):
        """One Uzawa step of the oracle on the window, boundary velocities
        held: u (3, n_free), p (n,).  The colours are the cube's only if the
        origin's coordinate sum is a multiple of 4."""
        from oracle import multigrid as MG
        assert int(self.origin.sum()) % 4 == 0
        L = self.L
        H = MG.Hierarchy(levels={0: L}, coarsest=0, finest=0)
        col = MG.colour_of(L)
        H.colours_u[0] = [np.where(col[L.free] == c)[0] for c in range(4)]
        H.colours_p[0] = [np.where(col == c)[0] for c in range(4)]
        fl, gl = self.lift(u, f, g)
        uf, pp = u[L.free].T.copy(), np.array(p, dtype=float, copy=True)
        MG.uzawa_step(H, 0, uf, pp, fl, gl)
        return uf, pp
