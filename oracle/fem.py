"""Oracle: P1 element integrals and global assembly (test infrastructure).

Every matrix is assembled from element integrals over the fine tetrahedra of
one refinement level -- the plain definition of the discrete forms of the
variational problem in Sec. 2.1 (bilinear forms a_1, b, c_l and linear forms
f, g_l), with P1 hat functions phi_i whose gradients are constant per element:

  A[i,j]   = a_1(phi_j, phi_i) = nu * int grad phi_i . grad phi_j        (Laplace form)
  A2[a][b][i,j] = a_2(phi_j e_b, phi_i e_a) = 2 nu int D(phi_j e_b) : D(phi_i e_a)
           = nu int (delta_ab grad phi_i . grad phi_j + d_b phi_i d_a phi_j)   (D form,
             D(u) = (grad u + grad u^T) / 2; expanding D : D gives the two terms)
  B_d[i,j] = b(phi_j e_d, phi_i) = - int phi_i  d_d phi_j                 (rows: pressure)
  C[i,j]   = c_l(phi_i, phi_j) = sum_T delta h_T^2 int_T grad phi_i . grad phi_j,
             h_T = |T|^(1/3), delta = 1/12                                 (Sec. 2.1)
  M[i,j]   = int phi_i phi_j   (consistent mass), m_i = int phi_i (lumped)
  G_d[i,j] : g_l(phi_i) for f = sum_j f_j phi_j e_d, i.e.
             g_l(phi_i) = - sum_T delta h_T^2 int_T f . grad phi_i  (Sec. 2.1)
             G_d[i,j] = - sum_{T ∋ i,j} delta h_T^2 (|T|/4) d_d phi_i|_T

With the barycentric functions lambda_m of T: int_T phi_m = |T|/4 and
int_T phi_m phi_n = |T| (1 + [m == n]) / 20.

All matrices are n_nodes x n_nodes over every node of the level (boundary
nodes included); Dirichlet elimination happens in oracle.stokes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .mesh import RefinedMesh


@dataclass
class Operators:
    A: sp.csr_matrix
    B: list          # [B_0, B_1, B_2]
    C: sp.csr_matrix
    M: sp.csr_matrix
    m: np.ndarray    # lumped mass
    G: list          # [G_0, G_1, G_2]
    w_out: np.ndarray  # (n, 3): int over outflow faces of phi_i * n  (outflow functional)
    A2: list = None   # [[A2[a][b]]]: the D-form velocity blocks (row component a, column component b)


def element_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Volumes (nT,) and barycentric gradients (nT, 4, 3) of every tetrahedron."""
    X = xyz[tets]                                    # (nT, 4, 3)
    mat = np.concatenate([np.ones(X.shape[:2] + (1,)), X], axis=2)  # rows [1, x_v]
    coef = np.linalg.inv(mat)                        # column m: coefficients of lambda_m
    grads = np.transpose(coef[:, 1:, :], (0, 2, 1))  # (nT, m, 3)
    vol = np.abs(np.linalg.det(mat)) / 6.0
    return vol, grads


def _assemble(tets: np.ndarray, local: np.ndarray, n: int) -> sp.csr_matrix:
    """Sum element matrices local (nT, 4, 4) into an n x n CSR matrix."""
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    return sp.coo_matrix((local.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def assemble(mesh: RefinedMesh, nu: float = 1.0, delta: float = 1.0 / 12.0) -> Operators:
    n = mesh.n_nodes
    vol, grads = element_geometry(mesh.xyz, mesh.tets)
    hT2 = vol ** (2.0 / 3.0)
    K = vol[:, None, None] * np.einsum("tmc,tnc->tmn", grads, grads)  # int grad.grad
    A = _assemble(mesh.tets, nu * K, n)
    C = _assemble(mesh.tets, (delta * hT2)[:, None, None] * K, n)
    eye = np.eye(4)
    Mloc = (vol / 20.0)[:, None, None] * (1.0 + eye)[None]
    M = _assemble(mesh.tets, Mloc, n)
    m = np.bincount(mesh.tets.ravel(), weights=np.repeat(vol / 4.0, 4), minlength=n)
    B, G = [], []
    for d in range(3):
        # B_d[m, k] = -(|T|/4) d_d lambda_k  (independent of the test index m)
        Bl = -(vol / 4.0)[:, None, None] * np.broadcast_to(grads[:, None, :, d], (len(vol), 4, 4))
        B.append(_assemble(mesh.tets, Bl, n))
        # G_d[m, k] = -delta h_T^2 (|T|/4) d_d lambda_m  (independent of the force index k)
        Gl = -(delta * hT2 * vol / 4.0)[:, None, None] * np.broadcast_to(grads[:, :, None, d], (len(vol), 4, 4))
        G.append(_assemble(mesh.tets, Gl, n))
    # outflow functional weights: int_{Gamma_out} phi_i n dS (P1 on triangles: area/3 per vertex)
    w = np.zeros((n, 3))
    if len(mesh.outflow_tris):
        P = mesh.xyz[mesh.outflow_tris]
        area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
        for c in range(3):
            contrib = np.repeat((area / 3.0)[:, None] * mesh.outflow_normals[:, c][:, None], 3, axis=1)
            w[:, c] = np.bincount(mesh.outflow_tris.ravel(), weights=contrib.ravel(), minlength=n)
    # D form: nu int (delta_ab grad phi_m . grad phi_n + d_b phi_m d_a phi_n), m test (row), n trial (column)
    A2 = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            Kab = vol[:, None, None] * (grads[:, :, None, b] * grads[:, None, :, a])
            A2[a][b] = _assemble(mesh.tets, nu * ((K if a == b else 0.0) + Kab), n)
    return Operators(A=A, B=B, C=C, M=M, m=m, G=G, w_out=w, A2=A2)
