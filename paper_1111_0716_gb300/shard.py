"""Host-side decomposition of the exchange path over ranks.

Target k-points are independent units (each needs every occupied orbital of
every q): rank r applies V_x to the targets of a contiguous k-range and
computes its share of E_x with xx_energy_range; the shares are summed in rank
order so the total does not depend on the collective's reduction order.
"""
from __future__ import annotations

from typing import List, Tuple


def k_ranges(nk: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous (k_first, k_count) per rank, sizes differing by at most one."""
    if nk < 0 or world < 1:
        raise ValueError("bad decomposition")
    base, extra = divmod(nk, world)
    out, k0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k0, n))
        k0 += n
    return out


def fixed_order_sum(value: float, group=None) -> float:
    """Sum of one float per rank, added in rank order on every rank (FP64)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    world = dist.get_world_size(group)
    t = torch.tensor([float(value)], dtype=torch.float64)
    backend = dist.get_backend(group)
    if backend == "nccl":
        t = t.cuda()
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    total = 0.0
    for p in parts:
        total += float(p.item())
    return total
