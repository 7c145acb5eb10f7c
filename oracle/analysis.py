"""Oracle: the paper's cost models, evaluated (test infrastructure).

  * weighted operator count (Sec. 4.2, eq. "op_count"):
        n_op = n_I * sum_{l=0}^{L} 8^(l-L) n_op,l
    where n_op,l are the applications of one block on level l in one cycle;
  * memory model of the all-at-once multigrid (Sec. 4.1, eq. "memory"):
        m_t = 3 (n_u + n_p) sum_{l=0}^{L} 8^(l-L) * 8 bytes,
    and the variant without the finest right-hand side (Sec. 4.4);
  * free-DoF count of the unit cube: 3 (N-1)^3 velocity + (N+1)^3 pressure
    values at N = 2^k intervals per edge (Sec. 2.1 spaces, Tab. "itertime1");
  * work units of FMG with V_var(nu, nu) cycles (Sec. 5, eq. for E_TME): one
    smoothing step with its residual costs 13/10 WU, a cycle rooted at L
    applies 2 (nu + 2 (L - l)) steps on level l plus one residual per level,
    levels weighted by 8^(l - L), and the FMG runs cycles rooted at
    L, L-1, ..., weighted by 8^-k.
"""
from __future__ import annotations


def weighted_count(per_level: dict, finest: int, cycles: int) -> float:
    """cycles * sum_l 8^(l - L) * per_level[l]."""
    return cycles * sum(8.0 ** (l - finest) * n for l, n in per_level.items())


def memory_bytes(n_dofs: float, levels: int, rhs_on_the_fly: bool = False) -> float:
    """Memory model; ``levels`` = L + 1 grid levels (l = 0..L)."""
    L = levels - 1
    geo = sum(8.0 ** (l - L) for l in range(L + 1))
    if not rhs_on_the_fly:
        return 3.0 * n_dofs * geo * 8.0
    coarse = sum(8.0 ** (l - L) for l in range(L))
    return 2.0 * n_dofs * 8.0 + 3.0 * n_dofs * coarse * 8.0


def cube_free_dofs(level: int) -> int:
    n = 1 << level
    return 3 * (n - 1) ** 3 + (n + 1) ** 3


def fmg_work_units(finest: int, nu: int = 2, var_increment: int = 2, cycles: int = 1, coarsest: int = 1) -> float:
    """E_TME of Sec. 5: sum_{k=0}^{L-1} 8^-k sum_{l=1}^{L} 8^(l-L) (2 (nu + inc (L - l)) 13/10 + 1),
    times the cycles per level; levels counted from `coarsest` (the paper's l = 1)."""
    L = finest
    total = 0.0
    for k in range(L - coarsest + 1):
        for l in range(coarsest, L + 1):
            total += 8.0 ** (-k) * 8.0 ** (l - L) * (2 * (nu + var_increment * (L - l)) * 13.0 / 10.0 + 1.0)
    return cycles * total
