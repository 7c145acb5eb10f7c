"""Oracle: Krylov solvers of the coarse grid (test infrastructure).

Sec. 3.7: the all-at-once multigrid solves its coarsest level with MINRES on
the full saddle-point system, preconditioned block-diagonally as in Sec. 3.2
(the preconditioner diag(A_hat, S_hat)), where A_hat^{-1} is a CG solve on
each velocity block (relative accuracy 1e-3) and S_hat^{-1} is the inverse
lumped pressure mass.  Sec. 4.1: the serial cube runs use 5 coarse
iterations.

Both solvers start from the zero vector.  The stopping rules are written out
so the CUDA coarse solver can follow them step for step:
  * CG stops before an iteration when r.r <= rtol^2 * (r0.r0), or after
    max_iter iterations, or when d.Ad == 0;
  * MINRES stops after an iteration when |eta| <= rtol * gamma_1 (eta is the
    preconditioned residual norm carried by the recurrence), or after
    max_iter iterations.
"""
from __future__ import annotations

import numpy as np


def cg(apply_A, b: np.ndarray, max_iter: int, rtol: float) -> np.ndarray:
    """Plain conjugate gradients for an SPD operator, from x = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    d = r.copy()
    rr = float(np.dot(r, r))
    stop = rtol * rtol * rr
    for _ in range(max_iter):
        if rr <= stop or rr == 0.0:
            break
        q = apply_A(d)
        dq = float(np.dot(d, q))
        if dq == 0.0:
            break
        alpha = rr / dq
        x = x + alpha * d
        r = r - alpha * q
        rr_new = float(np.dot(r, r))
        beta = rr_new / rr
        d = r + beta * d
        rr = rr_new
    return x


def pminres(apply_K, b: np.ndarray, apply_Pinv, max_iter: int, rtol: float, history=None) -> np.ndarray:
    """Preconditioned MINRES from x = 0 (Lanczos three-term recurrence with
    Givens rotations), for a symmetric K and a symmetric positive preconditioner P.

    Recurrence (j = 1, 2, ...), with v_0 = w_0 = w_1 = 0, v_1 = b,
    z_1 = P^{-1} v_1, gamma_1 = sqrt(z_1 . v_1), gamma_0 = 1,
    c_0 = c_1 = 1, s_0 = s_1 = 0, eta = gamma_1:
        z_j     <- z_j / gamma_j
        delta_j  = (K z_j) . z_j
        v_{j+1}  = K z_j - (delta_j / gamma_j) v_j - (gamma_j / gamma_{j-1}) v_{j-1}
        z_{j+1}  = P^{-1} v_{j+1};   gamma_{j+1} = sqrt(z_{j+1} . v_{j+1})
        a0 = c_j delta_j - c_{j-1} s_j gamma_j
        a1 = sqrt(a0^2 + gamma_{j+1}^2)
        a2 = s_j delta_j + c_{j-1} c_j gamma_j
        a3 = s_{j-1} gamma_j
        c_{j+1} = a0 / a1;   s_{j+1} = gamma_{j+1} / a1
        w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j) / a1
        x_j     = x_{j-1} + c_{j+1} eta w_{j+1};   eta <- -s_{j+1} eta
    """
    x = np.zeros_like(b)
    v_prev = np.zeros_like(b)
    v = b.copy()
    z = apply_Pinv(v)
    gamma = float(np.sqrt(max(np.dot(z, v), 0.0)))
    if gamma == 0.0:
        return x
    gamma1 = gamma
    gamma_prev = 1.0
    eta = gamma
    c_prev, c = 1.0, 1.0
    s_prev, s = 0.0, 0.0
    w_prev = np.zeros_like(b)
    w = np.zeros_like(b)
    for _ in range(max_iter):
        z = z / gamma
        Kz = apply_K(z)
        delta = float(np.dot(Kz, z))
        v_next = Kz - (delta / gamma) * v - (gamma / gamma_prev) * v_prev
        z_next = apply_Pinv(v_next)
        gamma_next = float(np.sqrt(max(np.dot(z_next, v_next), 0.0)))
        a0 = c * delta - c_prev * s * gamma
        a1 = float(np.sqrt(a0 * a0 + gamma_next * gamma_next))
        a2 = s * delta + c_prev * c * gamma
        a3 = s_prev * gamma
        if a1 == 0.0:
            break
        c_next = a0 / a1
        s_next = gamma_next / a1
        w_next = (z - a3 * w_prev - a2 * w) / a1
        x = x + (c_next * eta) * w_next
        eta = -s_next * eta
        if history is not None:
            history.append(abs(eta) / gamma1)
        # shift
        v_prev, v = v, v_next
        z = z_next
        gamma_prev, gamma = gamma, gamma_next
        c_prev, c = c, c_next
        s_prev, s = s, s_next
        w_prev, w = w, w_next
        if abs(eta) <= rtol * gamma1 or gamma == 0.0:
            break
    return x
