"""Sharding of independent solve units (k-points, right-hand-side blocks) over ranks.

Every right-hand side is an independent multishift solve (the paper distributes k/q points
over "pools" and perturbations G' over "images", Sec. 2.10), so ranks share no data during
a solve: each rank takes its own units and only the timing is reduced.
"""
from __future__ import annotations


def units_for_step(step: int, world: int, rank: int, n_units: int) -> int:
    """Unit processed by `rank` at `step`: consecutive steps cycle over the units, and the
    ranks of one step take consecutive units (weak scaling: one unit per rank per step)."""
    if n_units < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("bad partition arguments")
    return (step * world + rank) % n_units


def block_range(n: int, world: int, rank: int) -> tuple:
    """Contiguous block [lo, hi) of n items for rank (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)
