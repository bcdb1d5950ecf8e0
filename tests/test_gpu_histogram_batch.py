"""GPU histogram and batched launch against the oracle (same inputs), and the
host-buffer end-to-end entry against the device one."""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _gpu_hist(nat, N, lw, n_bins, lo, hi, n_sub=1, id_offset=0):
    import torch
    tN = torch.from_numpy(np.ascontiguousarray(N)).cuda()
    tl = torch.from_numpy(np.ascontiguousarray(lw)).cuda()
    bins = nat.empty_bins(n_bins * n_sub)
    counts = nat.empty_counts(1)
    nat.fpt_histogram(tN, tl, n_bins, lo, hi, bins, counts, n_sub=n_sub, id_offset=id_offset)
    f, c = nat.bins_to_numpy(bins)
    return f.reshape(n_sub, n_bins, 7), c.reshape(n_sub, n_bins), counts.cpu().numpy()[0]


def _compare(f, c, cnt, ref_bins, ref_counts):
    assert np.array_equal(cnt, ref_counts)
    assert np.array_equal(c, ref_bins[..., 7].astype(np.int64))
    assert np.array_equal(f[..., 0], ref_bins[..., 0])  # max: exact
    # every sum adds terms of one sign (x = ln w - max <= 0), so each agrees to
    # rounding relative to itself; the order of the FP64 atomics is not fixed
    for k in range(1, 7):
        np.testing.assert_allclose(f[..., k], ref_bins[..., k], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("n,n_bins,n_sub", [(1, 10, 1), (1000, 7, 1), (100003, 400, 1),
                                            (65537, 100, 11), (200000, 4096, 1)])
def test_histogram_matches_oracle(nat, n, n_bins, n_sub):
    N, lw = W.random_records(n, seed=n, lo=7.0, hi=10.0)
    f, c, cnt = _gpu_hist(nat, N, lw, n_bins, 7.0, 10.0, n_sub=n_sub, id_offset=3)
    rb, rc = oracle.histogram(N, lw, n_bins, 7.0, 10.0, n_sub=n_sub, id_offset=3)
    _compare(f, c, cnt, rb, rc)


def test_histogram_concentrated_and_edge_cases(nat):
    # everything in two bins (drift-dominated shape): heavy same-bin aggregation
    rng = np.random.default_rng(1)
    N = 8.5 + 0.001 * rng.standard_normal(300000)
    lw = -50 + rng.standard_normal(300000)
    f, c, cnt = _gpu_hist(nat, N, lw, 400, 7.0, 10.0)
    rb, rc = oracle.histogram(N, lw, 400, 7.0, 10.0)
    _compare(f, c, cnt, rb, rc)
    # empty input, infinities, NaN, exact binary edges
    e = np.concatenate([np.arange(0, 9) / 8.0, [np.inf, np.nan, -1.0, 2.0]])
    f, c, cnt = _gpu_hist(nat, e, np.zeros(e.size), 8, 0.0, 1.0)
    rb, rc = oracle.histogram(e, np.zeros(e.size), 8, 0.0, 1.0)
    _compare(f, c, cnt, rb, rc)
    import torch
    bins = nat.empty_bins(8)
    counts = nat.empty_counts(1)
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    nat.fpt_histogram(z, z, 8, 0.0, 1.0, bins, counts)
    f, c = nat.bins_to_numpy(bins)
    assert np.all(c == 0) and np.all(f[:, 0] == -np.inf) and counts.cpu().tolist() == [[0, 0, 0, 0]]


@pytest.mark.parametrize("lo,hi,n_bins", [(7.0, 10.0, 400), (0.1, 0.7, 3), (-1.3, 2.9, 4095)])
def test_histogram_bin_edges_exact(nat, lo, hi, n_bins):
    """Records on the bin edges lo + k d of a non-dyadic width, and one and two
    ulp either side of them, land in the same bins as the oracle's division
    (the kernel multiplies by 1/d and divides only next to an edge)."""
    d = (hi - lo) / n_bins
    k = np.arange(n_bins + 1, dtype=np.float64)
    edges = np.concatenate([lo + k * d, k * d + lo, lo + (k + 0.5) * d, hi - (n_bins - k) * d])
    N = np.concatenate([edges, np.nextafter(edges, np.inf), np.nextafter(edges, -np.inf),
                        np.nextafter(np.nextafter(edges, np.inf), np.inf),
                        np.nextafter(np.nextafter(edges, -np.inf), -np.inf)])
    lw = np.random.default_rng(n_bins).normal(-3.0, 2.0, N.size)
    f, c, cnt = _gpu_hist(nat, N, lw, n_bins, lo, hi)
    rb, rc = oracle.histogram(N, lw, n_bins, lo, hi)
    _compare(f, c, cnt, rb, rc)


def test_histogram_rejects_bad_arguments(nat):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    bins = nat.empty_bins(8)
    counts = nat.empty_counts(1)
    for args in ((0, 0.0, 1.0, 1), (8, 1.0, 1.0, 1), (8, 0.0, math.inf, 1), (4097, 0.0, 1.0, 1),
                 (8, 0.0, 1.0, 0), (1024, 0.0, 1.0, 5)):
        with pytest.raises(nat.FptError) as ei:
            nat.fpt_histogram(x, x, args[0], args[1], args[2], bins, counts, n_sub=args[3])
        assert ei.value.code == nat.FPT_EINVAL


def test_batch_equals_individual_calls_and_histograms(nat):
    """A batched launch of several sets (uneven lengths, some with a wall) gives
    the same records as one call per set, and its histograms are those of its
    own records (same inputs to the oracle histogram)."""
    import torch
    wl = W.batched_uneven(scale=1 / 512)  # 64 sets x 2048 runs
    wl.precision = "f32_kahan"
    specs = wl.sets[::7]  # 10 sets spanning phi_in, m, b
    specs[1].phi_uv = specs[1].phi_in * 1.05
    sub = W.Workload("sub", specs, "f32_kahan", seed=3)
    N, lw, bins, counts = nat.simulate_workload(sub)
    N = N.cpu().numpy()
    lw = lw.cpu().numpy()
    f, c = nat.bins_to_numpy(bins)
    cnt = counts.cpu().numpy()
    off = 0
    boff = 0
    for i, s in enumerate(specs):
        one = W.Workload("one", [s], "f32_kahan", seed=3)
        N1, lw1, _, _ = nat.simulate_workload(one, with_hist=False)
        assert np.array_equal(N[off: off + s.n_traj], N1.cpu().numpy())
        assert np.array_equal(lw[off: off + s.n_traj], lw1.cpu().numpy())
        rb, rc = oracle.histogram(N[off: off + s.n_traj], lw[off: off + s.n_traj], s.n_bins,
                                  s.hist_lo, s.hist_hi)
        _compare(f[boff: boff + s.n_bins][None], c[boff: boff + s.n_bins][None], cnt[i], rb, rc)
        off += s.n_traj
        boff += s.n_bins


def test_host_entry_matches_device_entry(nat):
    import torch
    wl = W.drift_dominated_ladder(scale=1 / 1024)
    N, lw, bins, counts = nat.simulate_workload(wl)
    sets = nat.make_sets(wl.sets)
    n = wl.n_total
    hN = torch.empty(n, dtype=torch.float64).pin_memory()
    hl = torch.empty(n, dtype=torch.float64).pin_memory()
    hb = torch.empty((sum(s.n_bins for s in wl.sets), nat.BIN_FIELDS), dtype=torch.float64)
    hc = torch.empty((len(wl.sets), 4), dtype=torch.int64)
    s0 = wl.sets[0]
    p = nat.make_params(precision=wl.precision, m=s0.m, n_max=s0.n_max)
    nat.fpt_simulate_batch_host(p, sets, wl.seed, hN, hl, hb, hc)
    assert torch.equal(hN, N.cpu()) and torch.equal(hl, lw.cpu())
    assert torch.equal(hc, counts.cpu())
    # counts and maxima are exact; the FP64 sums are accumulated with atomics,
    # so their last bits depend on the order the GPU happens to add them in
    fb, cb = nat.bins_to_numpy(bins)
    fh, ch = nat.bins_to_numpy(hb)
    assert np.array_equal(cb, ch) and np.array_equal(fb[:, 0], fh[:, 0])
    np.testing.assert_allclose(fh[:, 1:], fb[:, 1:], rtol=1e-12, atol=1e-300)
    # the records are copied on a second stream while the histogram runs: the
    # same results with pageable record buffers, and on a caller's stream
    for pinned, on_stream in ((False, False), (True, True)):
        hN2 = torch.full((n,), -1.0, dtype=torch.float64)
        hl2 = torch.full((n,), -1.0, dtype=torch.float64)
        if pinned:
            hN2, hl2 = hN2.pin_memory(), hl2.pin_memory()
        hb2, hc2 = torch.empty_like(hb), torch.empty_like(hc)
        s = torch.cuda.Stream() if on_stream else None
        p2 = nat.make_params(precision=wl.precision, m=s0.m, n_max=s0.n_max, stream=s)
        nat.fpt_simulate_batch_host(p2, sets, wl.seed, hN2, hl2, hb2, hc2)
        assert torch.equal(hN2, hN) and torch.equal(hl2, hl) and torch.equal(hc2, hc)
        fh2, ch2 = nat.bins_to_numpy(hb2)
        assert np.array_equal(ch2, ch) and np.array_equal(fh2[:, 0], fh[:, 0])
        np.testing.assert_allclose(fh2[:, 1:], fh[:, 1:], rtol=1e-12, atol=1e-300)


def test_invalid_arguments_are_rejected_before_launch(nat):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    bad = [dict(dN=0.0), dict(dN=math.nan), dict(phi_uv=2.0), dict(n_max=math.inf),
           dict(n_max=1e7, dN=1e-6)]
    for kw in bad:
        args = dict(phi_in=3.0, phi_end=math.sqrt(2), phi_uv=math.inf, dN=1e-3, n_max=6.0)
        args.update(kw)
        p = nat.make_params(precision="f64", m=1.0, n_max=args.pop("n_max"))
        with pytest.raises(nat.FptError) as ei:
            nat.fpt_simulate(p, 8, args["phi_in"], args["phi_end"], args["phi_uv"], args["dN"], 1.0, 0,
                             x, x)
        assert ei.value.code == nat.FPT_EINVAL
    p = nat.make_params(precision="f32_kahan", m=1.0, n_max=6.0, k_steps=12)
    with pytest.raises(nat.FptError):
        nat.fpt_simulate(p, 8, 3.0, math.sqrt(2), math.inf, 1e-3, 1.0, 0, x, x)


def test_graph_plan_reproduces_batched_call(nat):
    """The graph-captured plan equals fpt_simulate_batch for two seeds in a row."""
    import torch
    wl = W.batched_uneven(scale=1 / 1024)
    specs = wl.sets[::4]
    sets = nat.make_sets(specs)
    n = sum(s.n_traj for s in specs)
    nb = sum(s.n_bins for s in specs)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    bins = nat.empty_bins(nb)
    counts = nat.empty_counts(len(specs))
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = nat.make_params(precision="f32_kahan", m=1.0, n_max=10.0, k_steps=32, steps_out=steps)
    plan = nat.Plan(p, sets, N, lw, bins, counts)
    for seed in (5, 6):
        steps.zero_()
        plan.launch(seed)
        got = (N.clone(), lw.clone(), counts.clone(), int(steps.item()))
        f_plan, c_plan = nat.bins_to_numpy(bins)
        steps.zero_()
        q = nat.make_params(precision="f32_kahan", m=1.0, n_max=10.0, k_steps=32, steps_out=steps)
        N2 = torch.empty_like(N)
        l2 = torch.empty_like(lw)
        b2 = nat.empty_bins(nb)
        c2 = nat.empty_counts(len(specs))
        nat.fpt_simulate_batch(q, sets, seed, N2, l2, b2, c2)
        assert torch.equal(got[0], N2) and torch.equal(got[1], l2) and torch.equal(got[2], c2)
        assert got[3] == int(steps.item())
        f2, cc2 = nat.bins_to_numpy(b2)
        assert np.array_equal(c_plan, cc2) and np.array_equal(f_plan[:, 0], f2[:, 0])
    plan.close()
