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
    """A block of (2^wl + 1)^3 nodes of the unit cube's Kuhn lattice at
    `level`, from lattice coordinates `origin`, assembled by the oracle: its
    refinement of the unit cube at level wl (the same Kuhn lattice, which
    is invariant under lattice translations), scaled to the spacing
    2^-level and moved to the origin.  Every row of an interior node of the
    window is the row of the whole cube at that node, so the oracle can
    produce sampled outputs of levels it cannot assemble.

    The window's boundary nodes are Dirichlet nodes of its oracle level.
    Where they lie on the cube's boundary they are Dirichlet nodes of the
    cube too; elsewhere (the "held" faces) they stand for nodes whose rows
    reach outside the window and keep the values they are given."""

    def __init__(self, level, origin, wl):
        from oracle import mesh as OM
        from oracle import stokes as S
        cube = W.unit_cube()
        m = OM.refine(cube.vertices, cube.tets, cube.bc_flags, wl)
        scale = 2.0 ** (wl - level)
        m.xyz = m.xyz * scale + np.asarray(origin, float) / (1 << level)
        m.h = m.h * scale
        self.level, self.wl = level, wl
        self.origin = np.asarray(origin, np.int64)
        self.L = S.build_level(m)
        self.ijk = m.ijk
        self.glob = m.ijk + self.origin
        d = (1 << level) + 1
        self.index = self.glob[:, 0] + d * (self.glob[:, 1] + d * self.glob[:, 2])
        self.on_cube_boundary = ((self.glob == 0) | (self.glob == (1 << level))).any(axis=1)
        self.coords = self.glob / float(1 << level)
        n = 1 << wl
        held = np.full(len(self.glob), np.iinfo(np.int64).max)
        for a in range(3):
            if self.origin[a] > 0:
                held = np.minimum(held, self.ijk[:, a])
            if self.origin[a] + n < (1 << level):
                held = np.minimum(held, n - self.ijk[:, a])
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
