"""Source sharding over independent replicas (one process per GPU).

The TSM sources are independent (Sec. 2.1-2.2: each noise vector is solved and
contracted on its own), so several GPUs split the source index range and
exchange nothing until the end, when the per-source loops are gathered to
rank 0 in rank order and combined once (the same combine kernel as a single
process, so the result is bit-identical for any number of replicas).

Weak scaling: every rank owns N_HP HP sources and N_LP LP sources; the global
HP set is [0, world * N_HP) and the LP set follows it.
"""
import numpy as np


def source_ranges(n_hp, n_lp, rank, world):
    """(hp_range, lp_range) of global source indices owned by `rank` (weak scaling)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    hp = (rank * n_hp, (rank + 1) * n_hp)
    lp0 = world * n_hp
    lp = (lp0 + rank * n_lp, lp0 + (rank + 1) * n_lp)
    return hp, lp


def split_ranges(n_hp, n_lp, rank, world):
    """Strong-scaling split of a fixed [0, N_HP) + [N_HP, N_HP + N_LP) source set."""
    def part(n, off):
        lo = off + (n * rank) // world
        hi = off + (n * (rank + 1)) // world
        return lo, hi
    return part(n_hp, 0), part(n_lp, n_hp)


def gather_per_source(per_corr, per_lp, group=None):
    """Gather per-source loop arrays (numpy, complex128) to every rank in rank
    order with torch.distributed (gloo or NCCL via CPU tensors).  Returns the
    concatenated (per_corr, per_lp)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)

    def gather(arr):
        t = torch.from_numpy(np.ascontiguousarray(arr).view(np.float64))
        n = torch.tensor([t.shape[0]], dtype=torch.int64)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, n, group=group)
        mx = int(max(s.item() for s in sizes))
        pad = torch.zeros((mx,) + tuple(t.shape[1:]), dtype=t.dtype)
        pad[:t.shape[0]] = t
        outs = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(outs, pad, group=group)
        parts = [o[:int(s.item())].numpy() for o, s in zip(outs, sizes)]
        return np.concatenate(parts).view(np.complex128)

    return gather(per_corr), gather(per_lp)
