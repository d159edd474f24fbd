"""Sharding of independent solve units (k-points, right-hand-side blocks) over ranks.

Every right-hand side is an independent multishift solve (the paper distributes k/q points
over "pools" and perturbations G' over "images", Sec. 2.10), so ranks share no data during
a solve: each rank takes its own units and only the timing is reduced.  The one exchange
step after the solves is the k-point sum of the density response (Eq. 5): each rank
accumulates the contributions of its own k-points and allreduce_density sums them.
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


def allreduce_density(dn, group=None):
    """Sum a density-response accumulator dn[G][G'][omega] (a complex torch tensor, host or
    device, holding this rank's k-point contributions) over the ranks of `group`, in place,
    so every rank ends with the full k-point sum of Eq. 5.  A no-op without an initialised
    process group or with one rank.  The backend must support the tensor's device (gloo for
    host tensors, NCCL for CUDA tensors); complex values travel as their real pairs, so dn must
    be contiguous (a ValueError otherwise)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return dn
    if not dn.is_complex():
        raise TypeError("dn must be a complex tensor")
    if not dn.is_contiguous():
        raise ValueError("dn must be contiguous (reduce a contiguous copy and copy it back)")
    view = torch.view_as_real(dn)
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return dn
