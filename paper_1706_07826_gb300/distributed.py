"""Multi-GPU sharding of Multi-start SPVAR (Alg. 2).

The starts of Alg. 2 are independent, so a multi-GPU run gives each rank a
contiguous block of the global start indices.  Start s keeps counter word s
whatever rank runs it, so the sharded run computes exactly what one GPU would
compute.  Nothing is exchanged while sampling.  After a run, one MIN
all-reduce gives the best energy and one all-gather gives the per-start best
energies, which is all the R99/TTS99 success rate needs.
"""
import numpy as np


def shard_starts(num_starts, rank, world):
    """(first, count) of the global starts that `rank` runs: near-equal
    contiguous blocks, the first `num_starts % world` ranks one larger."""
    if world < 1 or not 0 <= rank < world or num_starts < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(num_starts, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def combine_best(local_best, group=None, device=None):
    """Global minimum of the best energies and every rank's per-start best
    energies in global start order.

    local_best: int64 array of this rank's per-start best energies (its
    shard, in order).  Returns (global_min, all_best)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = device if device is not None else torch.device("cpu")
    loc = torch.as_tensor(np.asarray(local_best, np.int64), device=dev)
    n = torch.tensor([loc.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(s.item() for s in sizes))
    pad = torch.full((m,), np.iinfo(np.int64).max, dtype=torch.int64, device=dev)
    pad[:loc.numel()] = loc
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    allb = np.concatenate([p[:int(s.item())].cpu().numpy() for p, s in zip(parts, sizes)])
    best = torch.tensor([int(loc.min().item()) if loc.numel() else np.iinfo(np.int64).max], dtype=torch.int64,
                        device=dev)
    dist.all_reduce(best, op=dist.ReduceOp.MIN, group=group)
    return int(best.item()), allb


def success_rate(all_best, e_known):
    """Fraction of starts whose best energy reaches e_known (Sec. III.A R99)."""
    a = np.asarray(all_best)
    return float((a <= e_known).mean()) if a.size else 0.0
