"""Multi-rank path on the CPU: two gloo ranks each simulate their shard of the
run ids (with the FP64 oracle standing in for a GPU) and merge histograms
through the library's fpt_hist_merge (host code, no GPU); the result equals
the one-process run exactly (records, counts, maxima) and to 1e-12 (sums)."""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import shard
from paper_2206_11234_gb300 import workloads as W

SPEC = dict(phi_in=3.0, m=1.0, b=0.8, dN=2e-3, n_max=6.0, n_traj=3001, phi_uv=3.6, hist_lo=0.0, hist_hi=6.0,
            n_bins=60)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(spec):
    r = oracle.make_run(m=spec.m, phi_in=spec.phi_in, phi_uv=spec.phi_uv, dN=spec.dN, b=spec.b, n_max=spec.n_max,
                        traj_offset=spec.traj_offset)
    N, lw, _ = oracle.simulate(r, spec.n_traj)
    bins, counts = oracle.histogram(N, lw, spec.n_bins, spec.hist_lo, spec.hist_hi, id_offset=spec.traj_offset)
    return N, lw, bins[0], counts


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    spec = W.SetSpec(**SPEC)
    mine = shard.shard_sets([spec], rank, world)[0]
    N, lw, bins, counts = _run(mine)
    mb, mc = shard.allgather_merge(shard.pack_bins(bins[:, :7], bins[:, 7]), counts)
    f = mb.numpy()[:, :7]
    c = mb.numpy().view(np.int64)[:, 7]
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), N=N, lw=lw, off=mine.traj_offset, f=f, c=c,
             cnt=counts, mc=mc.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    full = W.SetSpec(**SPEC)
    N, lw, bins, counts = _run(full)
    parts = [np.load(os.path.join(tmp_path, f"r{r}.npz")) for r in range(world)]
    # records: the shards are the one-process records, bit for bit
    cat_N = np.concatenate([p["N"] for p in parts])
    cat_lw = np.concatenate([p["lw"] for p in parts])
    assert np.array_equal(cat_N, N) and np.array_equal(cat_lw, lw)
    for p in parts:
        f, c = p["f"], p["c"]
        assert np.array_equal(c, bins[:, 7].astype(np.int64))
        assert np.array_equal(f[:, 0], bins[:, 0])
        np.testing.assert_allclose(f[:, 1:3], bins[:, 1:3], rtol=1e-12, atol=0)
        for k in range(3, 7):
            np.testing.assert_allclose(f[:, k], bins[:, k], rtol=1e-9, atol=1e-9 * np.abs(bins[:, k]).max())
    assert sum(int(p["cnt"][3]) for p in parts) == counts[3]
    for p in parts:
        assert np.array_equal(p["mc"], counts)


def test_shard_ranges_partition_the_ids():
    spec = W.SetSpec(**SPEC)
    for world in (1, 2, 3, 8):
        shards = [shard.shard_sets([spec], r, world)[0] for r in range(world)]
        assert sum(s.n_traj for s in shards) == spec.n_traj
        starts = [s.traj_offset for s in shards]
        assert starts == sorted(starts) and starts[0] == 0
        for a, b in zip(shards, shards[1:]):
            assert a.traj_offset + a.n_traj == b.traj_offset
    with pytest.raises(ValueError):
        shard.shard_sets([spec], 2, 2)


def _merge(fields, counts):
    from paper_2206_11234_gb300 import native
    parts = np.stack([shard.pack_bins(f, c) for f, c in zip(fields, counts)])
    out, _ = native.fpt_hist_merge(parts)
    return out.numpy()[:, :7], out.numpy().view(np.int64)[:, 7]


def test_merge_handles_empty_bins():
    f1 = np.array([[-np.inf, 0, 0, 0, 0, 0, 0], [1.0, 2.0, 3.0, -1.0, 1.0, -1.0, 1.0]])
    f2 = np.array([[0.5, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0], [-np.inf, 0, 0, 0, 0, 0, 0]])
    f, c = _merge([f1, f2], [np.array([0, 2]), np.array([1, 0])])
    assert np.array_equal(c, [1, 2])
    assert f[0, 0] == 0.5 and f[0, 1] == 1.0 and f[1, 1] == 2.0
    assert np.array_equal(f[0, 3:], [0, 0, 0, 0]) and np.array_equal(f[1, 3:], [-1, 1, -1, 1])
    # a bin empty in every part stays empty
    fe, ce = _merge([f1[:1], f1[:1]], [np.array([0]), np.array([0])])
    assert fe[0, 0] == -np.inf and np.all(fe[0, 1:] == 0) and ce[0] == 0


def test_merge_recentres_moments():
    """Two parts with different maxima: the merged moments equal the moments
    of the pooled sample about the pooled maximum."""
    rng = np.random.default_rng(4)
    a, b = rng.normal(-3, 1, 50), rng.normal(1, 2, 70)

    def part(x):
        m = x.max()
        y = x - m
        return np.array([m, np.exp(y).sum(), np.exp(2 * y).sum(), y.sum(), (y ** 2).sum(), (y ** 3).sum(),
                         (y ** 4).sum()])
    f, c = _merge([part(a)[None], part(b)[None]], [np.array([50]), np.array([70])])
    np.testing.assert_allclose(f[0], part(np.concatenate([a, b])), rtol=1e-12)
    assert c[0] == 120


def test_merge_rejects_bad_bins():
    from paper_2206_11234_gb300 import native
    bad = np.stack([shard.pack_bins(np.array([[np.nan, 0, 0, 0, 0, 0, 0]]), np.array([1]))])
    with pytest.raises(native.FptError):
        native.fpt_hist_merge(bad)
    neg = np.stack([shard.pack_bins(np.array([[0.0, 1, 1, 0, 0, 0, 0]]), np.array([-1]))])
    with pytest.raises(native.FptError):
        native.fpt_hist_merge(neg)


def test_resume_from_a_checkpoint_equals_one_run():
    """Checkpoint / resume: a run split at id k (the checkpoint is the seed,
    the next id and the histogram so far) and resumed over ids [k, n) gives,
    after fpt_hist_merge, the histogram of the uninterrupted run: counts and
    maxima exactly, sums to rounding."""
    from paper_2206_11234_gb300 import native
    full = W.SetSpec(**SPEC)
    _, _, bins, counts = _run(full)
    k = 1234
    first = W.SetSpec(**{**SPEC, "n_traj": k})
    rest = W.SetSpec(**{**SPEC, "n_traj": full.n_traj - k})
    rest.traj_offset = k
    _, _, b1, c1 = _run(first)
    _, _, b2, c2 = _run(rest)
    parts = np.stack([shard.pack_bins(b[:, :7], b[:, 7]) for b in (b1, b2)])
    out, oc = native.fpt_hist_merge(parts, np.stack([c1, c2]))
    f, c = out.numpy()[:, :7], out.numpy().view(np.int64)[:, 7]
    assert np.array_equal(c, bins[:, 7].astype(np.int64)) and np.array_equal(f[:, 0], bins[:, 0])
    np.testing.assert_allclose(f[:, 1:3], bins[:, 1:3], rtol=1e-12, atol=0)
    assert np.array_equal(oc.numpy(), counts)
