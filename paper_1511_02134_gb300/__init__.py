"""GB300 all-at-once Uzawa multigrid solver for stabilised P1-P1 Stokes on
hierarchical hybrid grids (Gmeiner, Huber, John, Ruede, Wohlmuth,
arXiv:1511.02134) -- Python binding of the C ABI in include/hhg_stokes.h.

This module only marshals arguments to the CUDA library
``_lib/libhhg_stokes.so``; every step of the solver runs in its kernels.
There is no fallback: if the library is missing, loading it raises.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA), float64,
C-contiguous; outputs are numpy arrays unless an ``out`` tensor is given.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = ["Mesh", "Options", "HHGError", "lattice_classify", "library_path", "load_library",
           "MODE_FP64", "MODE_FP32_IR"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libhhg_stokes.so")

MODE_FP64 = 0
MODE_FP32_IR = 1

NODE_ACTIVE, NODE_VFREE, NODE_IRREG, NODE_DIRICHLET, NODE_OUTFLOW, NODE_SLIP = 1, 2, 4, 8, 16, 32
FIELD = {"U": 0, "P": 1, "F": 2, "G": 3, "RU": 4, "RP": 5}
OP = {"uzawa_step": 0, "vel_forward": 1, "vel_backward": 2, "vel_rhs": 3, "pres_rhs": 4,
      "pres_sweep": 5, "residual": 6, "restrict": 7, "prolong_add": 8, "coarse_solve": 9,
      "vcycle": 10, "project": 11, "vel_forward_f": 12, "pres_sweep_f": 13, "refine": 14, "cycle": 15,
      "fused_pass0": 16, "fused_pass1": 17, "fused_pass2": 18}
ERRORS = {0: "ok", -1: "HHG_EINVAL", -2: "HHG_EMESH", -3: "HHG_ENOMEM", -4: "HHG_EDIVERGED",
          -5: "HHG_EMAXIT", -6: "HHG_ECUDA", -7: "HHG_ESTATE"}


class HHGError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("delta", ctypes.c_double), ("omega", ctypes.c_double),
                ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32), ("var_increment", ctypes.c_int32),
                ("coarsest_level", ctypes.c_int32), ("coarse_minres_max", ctypes.c_int32),
                ("coarse_minres_rtol", ctypes.c_double), ("coarse_cg_max", ctypes.c_int32),
                ("coarse_cg_rtol", ctypes.c_double), ("use_graphs", ctypes.c_int32),
                ("fuse_coarse_levels", ctypes.c_int32), ("fuse_max_nodes", ctypes.c_int32),
                ("team_blocks", ctypes.c_int32), ("fused_min_nodes", ctypes.c_int32),
                ("ir_fixed_point", ctypes.c_int32), ("spec_max_nodes", ctypes.c_int32),
                ("colour_block_z", ctypes.c_int32), ("resident_node_lists", ctypes.c_int32),
                ("fused_tile_rows", ctypes.c_int32), ("wait_poll_limit", ctypes.c_int64),
                ("operator_form", ctypes.c_int32), ("colour_pairs", ctypes.c_int32),
                ("fused_wait_test", ctypes.c_int32), ("quad_min_nodes", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("r0", ctypes.c_double), ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("history", ctypes.c_double * 64), ("fx_rescales", ctypes.c_int32)]


@dataclass
class Stats:
    cycles: int
    status: int
    rel_residual: float
    r0: float
    seconds: float
    kernel_launches: int
    history: list
    fx_rescales: int = 0


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load the CUDA library (build it first with ``paper_1511_02134_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {_LIB_PATH} (run python -m paper_1511_02134_gb300.build)")
    L = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "hhg_default_options": (None, [P]),
        "hhg_create_mesh": (I32, [P, I64, P, I64, P, I32, P, P, P]),
        "hhg_destroy": (None, [P]),
        "hhg_strerror": (ctypes.c_char_p, [I32]),
        "hhg_last_error": (ctypes.c_char_p, [P]),
        "hhg_lattice_dims": (I32, [P, I32, P]),
        "hhg_num_nodes": (I32, [P, I32, P]),
        "hhg_num_dofs": (I32, [P, I32, P, P]),
        "hhg_node_coords": (I32, [P, I32, P]),
        "hhg_node_flags": (I32, [P, I32, P]),
        "hhg_outflow_weights": (I32, [P, I32, P]),
        "hhg_device_bytes": (I32, [P, P]),
        "hhg_set_rhs": (I32, [P, P, P]),
        "hhg_set_initial": (I32, [P, P, P]),
        "hhg_vcycle": (I32, [P, I32, P]),
        "hhg_solve": (I32, [P, D, I32, I32, P, P, P]),
        "hhg_get_solution": (I32, [P, P, P]),
        "hhg_fmg_solve": (I32, [P, P, P, I32, I32, I32, P, P, P]),
        "hhg_apply_operator": (I32, [P, I32, P, P, P, P]),
        "hhg_adjoint_gradient": (I32, [P, P, P, D, I32, I32, P, P]),
        "hhg_level_field": (I32, [P, I32, I32, I32, I32, P]),
        "hhg_level_op": (I32, [P, I32, I32, I32, I32]),
        "hhg_lattice_classify": (I32, [P, I64, P, I64, P, I32, P, P]),
        "hhg_assemble_operator_host": (I32, [P, I64, P, I64, P, I32, P, P, P, P, P, P, P, P]),
        "hhg_time_op": (I32, [P, I32, I32, I32, I32, P]),
        "hhg_kernel_launches": (I32, [P, P]),
        "hhg_allocations": (I32, [P, P]),
        "hhg_coarse_solve_noalloc": (I32, [P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch.Tensor (host or device)


def _is_tensor(a) -> bool:
    return type(a).__module__.startswith("torch")


def _as_f64(a, shape=None):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if shape is not None and a.size != int(np.prod(shape)):
            raise ValueError(f"expected {shape} values, got {a.shape}")
        return a
    # torch tensor
    if a.dtype != __import__("torch").float64 or not a.is_contiguous():
        raise ValueError("torch inputs must be contiguous float64 tensors")
    if shape is not None and a.numel() != int(np.prod(shape)):
        raise ValueError(f"expected {shape} values, got {tuple(a.shape)}")
    return a


def default_options() -> Options:
    o = Options()
    load_library().hhg_default_options(ctypes.byref(o))
    return o


def _macro_arrays(vertices, tets, bc_flags):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    T = np.ascontiguousarray(tets, dtype=np.int32)
    B = None if bc_flags is None else np.ascontiguousarray(bc_flags, dtype=np.uint8)
    return V, T, B


def lattice_classify(vertices, tets, bc_flags, level: int):
    """Host-only node classification of a level: (dims, flags) in lattice order."""
    L = load_library()
    V, T, B = _macro_arrays(vertices, tets, bc_flags)
    dims = np.zeros(3, np.int64)
    rc = L.hhg_lattice_classify(_ptr(V), len(V), _ptr(T), len(T), _ptr(B), level, _ptr(dims), None)
    if rc:
        raise HHGError(rc, L.hhg_last_error(None).decode())
    flags = np.zeros(int(np.prod(dims)), np.uint8)
    rc = L.hhg_lattice_classify(_ptr(V), len(V), _ptr(T), len(T), _ptr(B), level, _ptr(dims), _ptr(flags))
    if rc:
        raise HHGError(rc, L.hhg_last_error(None).decode())
    return tuple(int(d) for d in dims), flags


def assemble_operator_host(vertices, tets, bc_flags, level: int, options: Options | None = None, **opts):
    """Host-only CSR of the saddle-point matrix of a level as the kernels apply
    it (hhg_assemble_operator_host): (kptr, kcol, kval, vnode, pnode, pmass),
    the unknowns being the free velocity nodes (component by component), then
    the active pressure nodes, with the lattice index of each unknown's node
    and the lumped mass of each pressure unknown."""
    L = load_library()
    V, T, B = _macro_arrays(vertices, tets, bc_flags)
    o = default_options() if options is None else options
    for k, v in opts.items():
        setattr(o, k, v)
    sizes = np.zeros(3, np.int64)
    args = (_ptr(V), len(V), _ptr(T), len(T), _ptr(B), level, ctypes.byref(o), _ptr(sizes))
    rc = L.hhg_assemble_operator_host(*args, None, None, None, None, None, None)
    if rc:
        raise HHGError(rc, L.hhg_last_error(None).decode())
    rows, nnz, nvel = (int(v) for v in sizes)
    kptr, kcol = np.zeros(rows + 1, np.int32), np.zeros(nnz, np.int32)
    kval = np.zeros(nnz)
    vnode, pnode = np.zeros(nvel, np.int64), np.zeros(rows - 3 * nvel, np.int64)
    pmass = np.zeros(rows - 3 * nvel)
    rc = L.hhg_assemble_operator_host(*args, _ptr(kptr), _ptr(kcol), _ptr(kval), _ptr(vnode), _ptr(pnode),
                                      _ptr(pmass))
    if rc:
        raise HHGError(rc, L.hhg_last_error(None).decode())
    return kptr, kcol, kval, vnode, pnode, pmass


class Mesh:
    """A level hierarchy on the current CUDA device (hhg_create_mesh)."""

    def __init__(self, vertices, tets, bc_flags, finest_level: int, options: Options | None = None,
                 stream=None, **opts):
        L = load_library()
        self._lib = L
        o = default_options() if options is None else options
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        V, T, B = _macro_arrays(vertices, tets, bc_flags)
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(int(stream))
        rc = L.hhg_create_mesh(_ptr(V), len(V), _ptr(T), len(T), _ptr(B), finest_level, ctypes.byref(o), s,
                               ctypes.byref(h))
        if rc:
            raise HHGError(rc, L.hhg_last_error(None).decode())
        self._h = h
        self.finest = finest_level
        self.coarsest = o.coarsest_level

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.hhg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, allow=()):
        if rc and rc not in allow:
            raise HHGError(rc, self._lib.hhg_last_error(self._h).decode())
        return rc

    # -- geometry --
    def dims(self, level=None):
        d = np.zeros(3, np.int64)
        self._check(self._lib.hhg_lattice_dims(self._h, self._lvl(level), _ptr(d)))
        return tuple(int(x) for x in d)

    def num_nodes(self, level=None) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.hhg_num_nodes(self._h, self._lvl(level), ctypes.byref(n)))
        return n.value

    def num_dofs(self, level=None):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.hhg_num_dofs(self._h, self._lvl(level), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free_dofs(self, level=None) -> int:
        nv, np_ = self.num_dofs(level)
        return 3 * nv + np_

    def node_coords(self, level=None):
        out = np.zeros((self.num_nodes(level), 3))
        self._check(self._lib.hhg_node_coords(self._h, self._lvl(level), _ptr(out)))
        return out

    def node_flags(self, level=None):
        out = np.zeros(self.num_nodes(level), np.uint8)
        self._check(self._lib.hhg_node_flags(self._h, self._lvl(level), _ptr(out)))
        return out

    def outflow_weights(self, level=None):
        out = np.zeros((self.num_nodes(level), 3))
        self._check(self._lib.hhg_outflow_weights(self._h, self._lvl(level), _ptr(out)))
        return out

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        self._check(self._lib.hhg_device_bytes(self._h, ctypes.byref(b)))
        return b.value

    def _lvl(self, level):
        return self.finest if level is None else int(level)

    # -- solver --
    def set_rhs(self, f_nodal=None, u_dirichlet=None):
        n = self.num_nodes()
        f = _as_f64(f_nodal, (n, 3))
        d = _as_f64(u_dirichlet, (n, 3))
        self._check(self._lib.hhg_set_rhs(self._h, _ptr(f), _ptr(d)))

    def set_initial(self, u=None, p=None):
        n = self.num_nodes()
        u = _as_f64(u, (n, 3))
        p = _as_f64(p, (n,))
        self._check(self._lib.hhg_set_initial(self._h, _ptr(u), _ptr(p)))

    def vcycle(self, count: int = 1) -> float:
        r = ctypes.c_double()
        self._check(self._lib.hhg_vcycle(self._h, count, ctypes.byref(r)))
        return r.value

    def solve(self, tol=1e-8, max_cycles=50, mode=MODE_FP64, u_out=None, p_out=None, want_solution=True):
        """Returns (u, p, stats); u/p are None when want_solution is False."""
        n = self.num_nodes()
        if want_solution and u_out is None:
            u_out = np.zeros((n, 3))
        if want_solution and p_out is None:
            p_out = np.zeros(n)
        st = _Stats()
        rc = self._lib.hhg_solve(self._h, tol, max_cycles, mode, _ptr(u_out), _ptr(p_out), ctypes.byref(st))
        self._check(rc, allow=(-5,))
        return u_out, p_out, _stats(st)

    def fmg_solve(self, f_nodal=None, u_dirichlet=None, cycles=1, nu=2, mode=MODE_FP64, u_out=None, p_out=None,
                  want_solution=True):
        """Full multigrid with `cycles` V_var(nu, nu) cycles per level (hhg_fmg_solve);
        returns (u, p, stats), u/p None when want_solution is False."""
        n = self.num_nodes()
        f = _as_f64(f_nodal, (n, 3))
        d = _as_f64(u_dirichlet, (n, 3))
        if want_solution and u_out is None:
            u_out = np.zeros((n, 3))
        if want_solution and p_out is None:
            p_out = np.zeros(n)
        st = _Stats()
        self._check(self._lib.hhg_fmg_solve(self._h, _ptr(f), _ptr(d), cycles, nu, mode, _ptr(u_out), _ptr(p_out),
                                            ctypes.byref(st)))
        return u_out, p_out, _stats(st)

    def get_solution(self, u_out=None, p_out=None):
        n = self.num_nodes()
        u_out = np.zeros((n, 3)) if u_out is None else u_out
        p_out = np.zeros(n) if p_out is None else p_out
        self._check(self._lib.hhg_get_solution(self._h, _ptr(u_out), _ptr(p_out)))
        return u_out, p_out

    def apply_operator(self, u, p, level=None):
        lvl = self._lvl(level)
        n = self.num_nodes(lvl)
        u = _as_f64(u, (n, 3))
        p = _as_f64(p, (n,))
        ku, kp = np.zeros((n, 3)), np.zeros(n)
        self._check(self._lib.hhg_apply_operator(self._h, lvl, _ptr(u), _ptr(p), _ptr(ku), _ptr(kp)))
        return ku, kp

    def adjoint_gradient(self, ju=None, jp=None, tol=1e-10, max_cycles=60, mode=MODE_FP64, out=None):
        n = self.num_nodes()
        ju = _as_f64(ju, (n, 3))
        jp = _as_f64(jp, (n,))
        out = np.zeros((n, 3)) if out is None else out
        st = _Stats()
        rc = self._lib.hhg_adjoint_gradient(self._h, _ptr(ju), _ptr(jp), tol, max_cycles, mode, _ptr(out),
                                            ctypes.byref(st))
        self._check(rc, allow=(-5,))
        return out, _stats(st)

    # -- step-level hooks (parity tests) --
    def level_field(self, level, field, precision=0, value=None, out=None):
        """Read (value None) or write a field of one level, in lattice order.
        value and out: float64 numpy arrays or contiguous float64 torch tensors
        (host or device); a read goes into `out` if given, else into a new
        numpy array, and returns it."""
        n = self.num_nodes(level)
        nc = 3 if field in ("U", "F", "RU") else 1
        shape = (n, nc) if nc == 3 else (n,)
        if value is None:
            if out is None:
                buf = np.zeros(shape)
            else:
                buf = _as_f64(out, shape)
                if buf is not out:
                    raise ValueError("out must be a contiguous float64 array")
            self._check(self._lib.hhg_level_field(self._h, level, precision, FIELD[field], 0, _ptr(buf)))
            return buf
        buf = _as_f64(value if _is_tensor(value) else np.asarray(value), shape)
        self._check(self._lib.hhg_level_field(self._h, level, precision, FIELD[field], 1, _ptr(buf)))
        return None

    def level_op(self, level, op, precision=0, count=1):
        self._check(self._lib.hhg_level_op(self._h, level, precision, OP[op], count))

    def time_op(self, level, op, precision=0, reps=10) -> float:
        """Mean device milliseconds of one run of `op` (CUDA events on the mesh stream)."""
        ms = ctypes.c_double()
        self._check(self._lib.hhg_time_op(self._h, level, precision, OP[op], reps, ctypes.byref(ms)))
        return ms.value

    def coarse_solve_noalloc(self, f, g, u, p):
        """Coarse-grid correction of (u, p) in place without device allocation
        (hhg_coarse_solve_noalloc); arrays of the coarsest level."""
        n = self.num_nodes(self.coarsest)
        f = _as_f64(f, (n, 3))
        g = _as_f64(g, (n,))
        for a, shape in ((u, (n, 3)), (p, (n,))):
            if _as_f64(a, shape) is not a:
                raise ValueError("u and p must be contiguous float64 arrays (updated in place)")
        self._check(self._lib.hhg_coarse_solve_noalloc(self._h, _ptr(f), _ptr(g), _ptr(u), _ptr(p)))

    def kernel_launches(self) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.hhg_kernel_launches(self._h, ctypes.byref(n)))
        return n.value

    def allocations(self) -> int:
        """cudaMalloc / cudaMallocHost calls made for this mesh so far (hhg_allocations)."""
        n = ctypes.c_int64()
        self._check(self._lib.hhg_allocations(self._h, ctypes.byref(n)))
        return n.value


def _stats(st) -> Stats:
    return Stats(cycles=st.cycles, status=st.status, rel_residual=st.rel_residual, r0=st.r0,
                 seconds=st.seconds, kernel_launches=st.kernel_launches,
                 history=[st.history[i] for i in range(min(st.cycles + 1, 64))], fx_rescales=st.fx_rescales)
