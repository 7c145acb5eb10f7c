"""Oracle: exact discrete solution by a sparse direct solve (test infrastructure).

Solves the linear system of Sec. 3 (matrix K, right-hand side (f, g)) for one
level.  For pure-Dirichlet problems K is singular with null vector (0, 1)
(the pressure constant, Sec. 2); the system is then bordered with the
constraint sum_i m_i p_i = 0 (the discrete L^2_0 condition), which has a
unique solution when g is consistent.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from .stokes import StokesLevel, full_matrix


def solve_direct(L: StokesLevel, f: np.ndarray, g: np.ndarray):
    K = full_matrix(L)
    b = np.concatenate([f.ravel(), g])
    n = K.shape[0]
    if L.pure_dirichlet:
        e = np.zeros(n)
        e[3 * L.n_u:] = L.m
        Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
        x = sla.spsolve(Kb, np.concatenate([b, [0.0]]))[:n]
    else:
        x = sla.spsolve(K.tocsc(), b)
    return x[:3 * L.n_u].reshape(3, L.n_u), x[3 * L.n_u:]
