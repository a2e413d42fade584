"""Walker sharding across ranks and the one exchange step of the method.

Walkers are independent given the counter-based random streams (the streams
depend only on seed, global walker id and step), so ranks run disjoint
walker ranges of the same simulation with no communication on the data
path.  The only exchange is the final sum of a few kilobytes of FP64
partial sums (the signal numerators, sum of alpha, the moment sums); it is
gathered and added in rank order so the result does not depend on timing.
"""
from __future__ import annotations

import numpy as np


def shard_range(rank: int, world: int, n_walkers: int, weak: bool = False):
    """Global walker range [begin, end) of `rank`.  weak=True gives every rank
    n_walkers walkers of its own (per-GPU work fixed as ranks are added);
    otherwise the n_walkers walkers are split into contiguous near-equal parts."""
    if weak:
        return rank * n_walkers, (rank + 1) * n_walkers
    return (n_walkers * rank) // world, (n_walkers * (rank + 1)) // world


def pack_partials(num: np.ndarray, alpha_sum: float, moments: np.ndarray) -> np.ndarray:
    """One rank's reducible sums as a flat FP64 vector, exactly as the library
    returns them (rms_read_partials): the signal numerators sum alpha
    e^{-i phi}, sum alpha, the moment sums."""
    num = np.asarray(num, np.complex128).ravel()
    return np.concatenate([num.real, num.imag, [alpha_sum], np.asarray(moments, np.float64).ravel()])


def unpack_partials(v: np.ndarray, S_shape, m_shape):
    """(S, moments, sum alpha) from a merged vector; S = numerators / sum alpha
    is computed by the library (rms_normalise_partials)."""
    from .api import rms_normalise_partials
    n = int(np.prod(S_shape))
    num = (v[:n] + 1j * v[n:2 * n]).reshape(S_shape)
    asum = float(v[2 * n])
    mom = v[2 * n + 1:].reshape(m_shape)
    return rms_normalise_partials(num, asum), mom, asum


def merge_in_rank_order(parts) -> np.ndarray:
    """Sum of per-rank vectors, rank 0 first (fixed order)."""
    acc = np.zeros_like(parts[0])
    for p in parts:
        acc = acc + p
    return acc


def allreduce_partials(vec: np.ndarray, group=None) -> np.ndarray:
    """Gather every rank's partial vector and add them in rank order
    (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.ascontiguousarray(vec, np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return merge_in_rank_order([o.cpu().numpy() for o in out])
