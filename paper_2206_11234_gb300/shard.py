"""Host logic for running one workload on several GPUs (one process each).

Runs are independent (arXiv:2206.11234 §2.1), so a workload shards by run id:
rank r of W simulates a contiguous id range of every parameter set, and
because each run's noise is a function of (seed, set id, run id) the union of
the shards is bit-identical to the one-process result.  Nothing is exchanged
on the data path; the only reduction is the optional merge of the per-rank
weighted histograms, whose bins carry max-shifted sums (max ln w, sum w/e^max,
sum w^2/e^(2 max), sum x^k for k = 1..4 with x = ln w - max, count) and merge
by rescaling to the common maximum (binomial re-centring of the moments).
"""
import copy
import math
from typing import List, Sequence, Tuple

import numpy as np


def shard_sets(specs: Sequence, rank: int, world: int) -> list:
    """Copies of the set specs restricted to rank's contiguous id range."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    out = []
    for s in specs:
        lo = s.n_traj * rank // world
        hi = s.n_traj * (rank + 1) // world
        t = copy.copy(s)
        t.traj_offset = getattr(s, "traj_offset", 0) + lo
        t.n_traj = hi - lo
        out.append(t)
    return out


def merge_bins(fields: Sequence[np.ndarray], counts: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """Merge histograms of disjoint run sets.  fields[r]: float64 [..., 7] with
    (max_lw, s1, s2, l1, l2, l3, l4); counts[r]: int64 [...].  Empty bins have
    max_lw = -inf and zero sums."""
    F = np.stack([np.asarray(f, dtype=np.float64) for f in fields])
    C = np.stack([np.asarray(c, dtype=np.int64) for c in counts])
    mx = F[..., 0].max(axis=0)
    live = np.isfinite(F[..., 0])
    with np.errstate(invalid="ignore", over="ignore"):
        scale = np.where(live, np.exp(F[..., 0] - mx), 0.0)
        delta = np.where(live, F[..., 0] - mx, 0.0)  # <= 0: shift of each part's moments
    out = np.empty(F.shape[1:], dtype=np.float64)
    out[..., 0] = mx
    out[..., 1] = (F[..., 1] * scale).sum(axis=0)
    out[..., 2] = (F[..., 2] * scale * scale).sum(axis=0)
    # sum (x + delta)^k = sum_i C(k, i) delta^(k - i) sum x^i, with sum x^0 = count
    L = [C.astype(np.float64)] + [F[..., 2 + i] for i in range(1, 5)]
    for k in range(1, 5):
        acc = np.zeros_like(L[0])
        for i in range(k + 1):
            acc += math.comb(k, i) * delta ** (k - i) * L[i]
        out[..., 2 + k] = np.where(live, acc, 0.0).sum(axis=0)
    return out, C.sum(axis=0)


def allgather_merge(fields: np.ndarray, counts: np.ndarray, group=None) -> Tuple[np.ndarray, np.ndarray]:
    """Merge every rank's histogram with torch.distributed (any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    f = torch.from_numpy(np.ascontiguousarray(fields, dtype=np.float64))
    c = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.int64))
    fs = [torch.empty_like(f) for _ in range(world)]
    cs = [torch.empty_like(c) for _ in range(world)]
    dist.all_gather(fs, f, group=group)
    dist.all_gather(cs, c, group=group)
    return merge_bins([x.numpy() for x in fs], [x.numpy() for x in cs])
