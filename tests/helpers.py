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
