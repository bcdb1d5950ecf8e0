"""Host logic for running one workload on several GPUs (one process each).

Runs are independent (arXiv:2206.11234 §2.1), so a workload shards by run id:
rank r of W simulates a contiguous id range of every parameter set, and
because each run's noise is a function of (seed, set id, run id) the union of
the shards is bit-identical to the one-process result.  Nothing is exchanged
on the data path; the only reduction is the optional merge of the per-rank
weighted histograms, whose bins carry max-shifted sums (max ln w, sum w/e^max,
sum w^2/e^(2 max), sum x^k for k = 1..4 with x = ln w - max, count): they are
gathered here and merged by the library (fpt_hist_merge: rescaling to the
common maximum, binomial re-centring of the moments).
"""
import copy
from typing import Sequence

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


def pack_bins(fields: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """fpt_bin layout: float64 [n, 8] from fields [n, 7] and int64 counts [n]
    (the count stored as the bits of an int64)."""
    out = np.empty((np.asarray(fields).shape[0], 8), dtype=np.float64)
    out[:, :7] = fields
    out.view(np.int64)[:, 7] = np.asarray(counts, dtype=np.int64)
    return out


def allgather_merge(bins, counts=None, group=None):
    """Every rank's histogram gathered with torch.distributed and merged by
    the library's fpt_hist_merge.  bins: this rank's bins as a float64 tensor
    [n_bins, 8] in fpt_bin layout, on the device the process group's backend
    works on (CUDA for NCCL, CPU for gloo); counts: int64 [4] or None.
    Returns the merged (bins, counts) as host tensors on every rank."""
    import torch
    import torch.distributed as dist
    from . import native
    world = dist.get_world_size(group)
    b = torch.as_tensor(bins).contiguous()
    parts = [torch.empty_like(b) for _ in range(world)]
    dist.all_gather(parts, b, group=group)
    cparts = None
    if counts is not None:
        c = torch.as_tensor(counts).to(b.device).contiguous()
        cl = [torch.empty_like(c) for _ in range(world)]
        dist.all_gather(cl, c, group=group)
        cparts = torch.stack([x.cpu() for x in cl])
    return native.fpt_hist_merge(torch.stack([x.cpu() for x in parts]), cparts)
