"""Oracle: the paper's cost models, evaluated (test infrastructure).

  * weighted operator count (Sec. 4.2, eq. "op_count"):
        n_op = n_I * sum_{l=0}^{L} 8^(l-L) n_op,l
    where n_op,l are the applications of one block on level l in one cycle;
  * memory model of the all-at-once multigrid (Sec. 4.1, eq. "memory"):
        m_t = 3 (n_u + n_p) sum_{l=0}^{L} 8^(l-L) * 8 bytes,
    and the variant without the finest right-hand side (Sec. 4.4);
  * free-DoF count of the unit cube: 3 (N-1)^3 velocity + (N+1)^3 pressure
    values at N = 2^k intervals per edge (Sec. 2.1 spaces, Tab. "itertime1").
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
