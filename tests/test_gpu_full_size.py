"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times: the library's autotuned launch shape (pilot
on 2 % of the runs, seed 99) and one graph-captured fpt_plan launch of the
stepper over all sets plus the per-set histograms, seed 0.

* m = 1, phi_in = 3, b = 1, 16384 runs, binary64: every run against the oracle
  (same crossing step for all but 1e-6 of the runs, N and ln w to 1e-12).
* Drift-dominated ladder (5 x 2^22 runs), 64 uneven sets (64 x 2^20) and the
  diffusion-dominated workload with a wall (3 x 2^25), binary32 state: runs
  sampled over each set's whole id range (first, last, evenly spread and
  random ids) recomputed one by one by the oracle.  The binary32 path is not
  the binary64 path rounded, so a run agrees when its censoring matches, its N
  is within two steps and its ln w within the accumulated binary32 error plus
  one step's increment (a crossing decided one step apart); nearly all runs
  cross in the same step.  The few that do not are long runs (tens of
  thousands of steps and more): the random-walk rounding of the binary32 state,
  amplified by the flow towards phi_end, moves their crossing by a few steps,
  so every run must still lie within 1e-3 N of the oracle's.  Wrong counters
  or a wrong set would move N by sigma_N and ln w by b sqrt(dN M), far outside
  these bounds.
* Every per-set histogram against the oracle's histogram of the GPU's own
  records: counts and maxima exact; the sums within the rounding bound of a
  sum of same-signed terms in any order, (n - 1) u, plus a few ulp per term.
* Properties at any size: ln w = 0 exactly for unbiased sets; <N> of the
  unbiased drift-dominated set against Eq. (19) to 1e-3; E[w] = 1.
* The drift-dominated ladder in binary32 against the binary64 GPU path on the
  same runs, every bin (the reduced-precision bar: within 3 combined sigma).
* The learned-bias inference (2^26 runs) against the survival PDE, on
  sampled runs against the oracle running the same network, and bin by bin
  against 2^15 oracle runs of that network.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import analytic as A
import oracle
from paper_2206_11234_gb300 import workloads as W
from test_gpu_mlp_parity import assert_bins_agree, per_bin_z
from test_gpu_parity import assert_f64_parity

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    yield native
    native.fpt_autotune_reset()


def _bench_launch(nat, wl):
    """The benchmark's launch: autotune, then one fpt_plan launch (seed 0)."""
    import torch
    specs = wl.sets
    n = wl.n_total
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    bins = nat.empty_bins(sum(s.n_bins for s in specs))
    counts = nat.empty_counts(len(specs))
    sets = nat.make_sets(specs)
    s0 = specs[0]
    stream = torch.cuda.current_stream()

    def params():
        return nat.make_params(model=s0.model, precision=wl.precision, m=s0.m, a0=s0.a0, s0=s0.s0,
                               n_max=s0.n_max, stream=stream)
    shape = nat.fpt_autotune(params(), sets, seed=99, fraction=0.02)[:2]
    plan = nat.Plan(params(), sets, N, lw, bins, counts)
    plan.launch(wl.seed, stream)
    torch.cuda.synchronize()
    plan.close()
    f, c = nat.bins_to_numpy(bins)
    return N.cpu().numpy(), lw.cpu().numpy(), f, c, counts.cpu().numpy(), shape


def _check_histograms(specs, N, lw, f, c, cnt):
    off = boff = 0
    for i, s in enumerate(specs):
        rb, rc = oracle.histogram(N[off:off + s.n_traj], lw[off:off + s.n_traj], s.n_bins, s.hist_lo, s.hist_hi)
        fb, cb = f[boff:boff + s.n_bins], c[boff:boff + s.n_bins]
        assert np.array_equal(cnt[i], rc) and cnt[i][3] == s.n_traj, i
        assert np.array_equal(cb, rb[0, :, 7].astype(np.int64)), i
        assert np.array_equal(fb[:, 0], rb[0, :, 0]), i
        rtol = 2.0 * (cb + 4) * U
        for k in range(1, 7):
            err = np.abs(fb[:, k] - rb[0, :, k])
            assert np.all(err <= rtol * np.abs(rb[0, :, k]) + 1e-300), (i, k, np.max(err / (np.abs(rb[0, :, k]) + 1e-300)))
        off += s.n_traj
        boff += s.n_bins


def _sample_ids(n, k, seed):
    rng = np.random.default_rng(seed)
    ids = np.concatenate([[0, n - 1], np.linspace(0, n - 1, k // 2).astype(np.int64),
                          rng.integers(0, n, k - k // 2 - 2)])
    return np.unique(ids)


def _oracle_runs(wl, samples):
    """samples: [(set index, run index within the set)] -> (N, lw, steps)."""
    def one(job):
        si, i = job
        s = wl.sets[si]
        r = oracle.make_run(model=s.model, m=s.m, a0=s.a0, s0=s.s0, phi_in=s.phi_in, phi_end=s.phi_end,
                            phi_uv=s.phi_uv, dN=s.dN, b=s.b, n_max=s.n_max, seed=wl.seed, set_id=s.set_id,
                            traj_offset=s.traj_offset + int(i))
        No, lo, so = oracle.simulate(r, 1)
        return No[0], lo[0], so[0]
    with ThreadPoolExecutor(16) as ex:
        out = list(ex.map(one, samples))
    return np.array([o[0] for o in out]), np.array([o[1] for o in out]), np.array([o[2] for o in out])


def _check_sampled_f32(wl, N, lw, per_set, seed):
    samples, gN, glw = [], [], []
    off = 0
    for si, s in enumerate(wl.sets):
        for i in _sample_ids(s.n_traj, per_set, seed + si):
            samples.append((si, i))
            gN.append(N[off + i])
            glw.append(lw[off + i])
        off += s.n_traj
    gN, glw = np.array(gN), np.array(glw)
    oN, olw, osteps = _oracle_runs(wl, samples)
    b = np.array([wl.sets[si].b for si, _ in samples])
    dN = np.array([wl.sets[si].dN for si, _ in samples])
    # unbiased sets: ln w is exactly zero on both sides
    assert np.all(glw[b == 0] == 0.0) and np.all(olw[b == 0] == 0.0)
    same_status = np.isinf(gN) == np.isinf(oN)
    fin = np.isfinite(gN) & np.isfinite(oN)
    dn = np.where(fin, np.abs(np.where(fin, gN, 0.0) - np.where(fin, oN, 0.0)), 0.0)
    dl = np.abs(glw - olw)
    # binary32 normals differ from binary64 ones by ~1e-6 with random sign, so
    # the sum over M steps drifts by ~1e-6 sqrt(M); a crossing one step apart
    # adds one increment, |b sqrt(dN) xi| + b^2 dN / 2 with |xi| < 6
    inc = b * np.sqrt(dN)
    lw_tol = inc * (1e-4 * np.sqrt(osteps) + 6.0) + 0.5 * b * b * dN + 1e-12
    agree = same_status & (~fin | (dn <= 2 * dN)) & (dl <= lw_tol)
    same_step = fin & (dn < dN)
    stats = dict(samples=len(samples), status_agree=float(same_status.mean()), agree=float(agree.mean()),
                 finite=int(fin.sum()), same_step=float(same_step.sum() / max(1, fin.sum())),
                 median_dN_over_dN=float(np.median(dn[fin] / dN[fin])) if fin.any() else 0.0,
                 median_dlw=float(np.median(dl[b > 0])) if (b > 0).any() else 0.0)
    print(wl.name, stats)
    for j in np.nonzero(~agree)[0][:40]:
        si, i = samples[j]
        st = wl.sets[si]
        print(f"  differs: set {si} (phi_in {st.phi_in:.3f}, m {st.m}, b {st.b}) run {i}: N {gN[j]!r} vs {oN[j]!r}, "
              f"ln w {glw[j]!r} vs {olw[j]!r}, oracle steps {osteps[j]}")
    assert same_status.mean() >= 0.995, stats
    assert np.all(dn[fin] <= 2 * dN[fin] + 1e-3 * oN[fin]), np.max(dn[fin] / oN[fin])
    assert agree.mean() >= 0.99, stats
    if fin.sum() >= 50:
        assert stats["same_step"] >= 0.95, stats
        assert stats["median_dN_over_dN"] <= 0.1, stats
    biased = b > 0
    if biased.any():
        assert np.median(dl[biased]) <= np.median((inc * 1e-5 * np.sqrt(osteps))[biased]) + 1e-9, stats
    return stats


def test_quadratic_b1_every_run_binary64(nat):
    wl = W.quadratic_fixed_b()
    N, lw, f, c, cnt, shape = _bench_launch(nat, wl)
    s = wl.sets[0]
    r = oracle.make_run(m=s.m, phi_in=s.phi_in, dN=s.dN, b=s.b, n_max=s.n_max, seed=wl.seed)
    No, lo, so = oracle.simulate(r, s.n_traj)
    assert_f64_parity(N, lw, No, lo, so, s.b, s.dN)
    _check_histograms(wl.sets, N, lw, f, c, cnt)
    print("quadratic b=1 launch shape", shape)


def test_drift_ladder_full_size(nat):
    wl = W.drift_dominated_ladder()
    N, lw, f, c, cnt, shape = _bench_launch(nat, wl)
    _check_sampled_f32(wl, N, lw, per_set=1000, seed=11)
    _check_histograms(wl.sets, N, lw, f, c, cnt)
    n = wl.sets[0].n_traj
    # unbiased set: every run finishes; <N> against Eq. (19) (quadrature)
    N0 = N[:n]
    assert np.all(np.isfinite(N0))
    ref = A.mean_fpt_quad(6.0, 0.01)
    assert abs(N0.mean() / ref - 1) < 1e-3, (N0.mean(), ref)
    # b = 0.5: E[w] = 1 (Var ln w = b^2 N ~ 2, well sampled by 2^22 runs)
    w = np.exp(lw[n:2 * n])
    assert abs(w.mean() - 1) < 4 * w.std() / math.sqrt(n), w.mean()
    print("drift ladder launch shape", shape)


def test_batched_uneven_full_size(nat):
    wl = W.batched_uneven()
    N, lw, f, c, cnt, shape = _bench_launch(nat, wl)
    _check_sampled_f32(wl, N, lw, per_set=64, seed=12)
    _check_histograms(wl.sets, N, lw, f, c, cnt)
    print("batched uneven launch shape", shape)


def test_diffusion_wall_full_size(nat):
    wl = W.diffusion_wall()
    N, lw, f, c, cnt, shape = _bench_launch(nat, wl)
    _check_sampled_f32(wl, N, lw, per_set=256, seed=13)
    _check_histograms(wl.sets, N, lw, f, c, cnt)
    print("diffusion wall launch shape", shape)


def test_drift_ladder_binary32_against_binary64_every_bin(nat):
    """The reduced-precision bar at full size: the drift-dominated ladder
    (5 x 2^22 runs, 400 bins per set) in binary32 + compensated log-weight
    against the binary64 GPU path on the same runs.  <N> agrees to 1e-3 (in
    fact ~1e-7); every bin with >= 400 runs agrees within 3 combined standard
    errors, the two estimates treated as independent (they share their noise,
    so this is loose: measured at most 0.18), and within 3 paired standard
    errors (the spread of the per-run differences, the resolution at which a
    systematic shift from binary32 arithmetic would show), the count beyond 3
    at most the 99.9 % binomial quantile and none beyond 5; per run, N differs
    by ~2e-5 (1e-3 sigma_N) and never by a whole step."""
    import torch
    wl32 = W.drift_dominated_ladder()
    wl64 = W.drift_dominated_ladder(precision="f64")
    N32, lw32, b32, c32 = nat.simulate_workload(wl32)
    N64, lw64, b64, c64 = nat.simulate_workload(wl64)
    torch.cuda.synchronize()
    n = wl32.sets[0].n_traj
    f32, k32 = nat.bins_to_numpy(b32)
    f64, k64 = nat.bins_to_numpy(b64)
    N32, N64 = N32.cpu().numpy(), N64.cpu().numpy()
    assert np.all(np.isfinite(N32)) and np.all(np.isfinite(N64))
    dn = np.abs(N32 - N64)
    print("|N32 - N64| quantiles 0.5 / 0.99 / 0.9999 / max:", np.quantile(dn, [0.5, 0.99, 0.9999]), dn.max(),
          "runs above 0.02 sigma:", int(np.sum(dn > 0.02 * 0.0203)))
    lw_d = np.abs(lw32.cpu().numpy() - lw64.cpu().numpy())
    print("|lw32 - lw64| quantiles 0.5 / 0.99 / 0.9999 / max:", np.quantile(lw_d, [0.5, 0.99, 0.9999]), lw_d.max())
    # binary32 rounding drifts N by ~2e-5 (1e-3 sigma_N); no run crosses more
    # than a step apart (|dN| < dN = 1e-3, measured max 5.6e-4), and ln w then
    # differs by that step's increment b sqrt(dN) |xi| < 6 b sqrt(dN)
    assert np.quantile(dn, 0.9999) < 0.01 * 0.0203 and dn.max() < 1e-3
    assert np.median(lw_d) < 1e-4 and lw_d.max() < 6 * 4.0 * math.sqrt(1e-3)
    from scipy.stats import binom
    worst, paired = [], []
    for s in range(len(wl32.sets)):
        sl = slice(s * n, (s + 1) * n)
        assert abs(N32[sl].mean() / N64[sl].mean() - 1) < 1e-3
        bs = slice(s * 400, (s + 1) * 400)
        P = []
        for f, k in ((f32[bs], k32[bs]), (f64[bs], k64[bs])):
            mx = f[:, 0]
            with np.errstate(over="ignore", invalid="ignore"):
                s1 = np.where(k > 0, np.exp(mx) * f[:, 1], 0.0)
                s2 = np.where(k > 0, np.exp(2 * mx) * f[:, 2], 0.0)
            p = s1 / (0.0075 * n)
            se = np.sqrt(np.maximum(s2 / n - (s1 / n) ** 2, 0.0) / n) / 0.0075
            P.append((p, se, k))
        (p1, e1, k1), (p2, e2, k2) = P
        use = (k1 >= 400) & (k2 >= 400)
        z = np.abs(p1[use] - p2[use]) / np.hypot(e1[use], e2[use])
        worst.append(float(z.max()))
        assert use.sum() >= 10
        assert np.all(z <= 3.0), (s, z.max())
        # paired: both precisions ran the same runs, so the standard error of the
        # difference is that of the per-run differences of the bin's weighted
        # indicator, sqrt(var_i(w32_i 1{i in j under binary32} - w64_i 1{i in j
        # under binary64}) / n) / d -- orders of magnitude below the combined
        # one, and the bar at which a systematic binary32 shift would show
        j32 = np.clip(np.ceil((N32[sl] - 7.0) / 0.0075).astype(np.int64) - 1, -1, 400)
        j64 = np.clip(np.ceil((N64[sl] - 7.0) / 0.0075).astype(np.int64) - 1, -1, 400)
        w32 = np.exp(lw32.cpu().numpy()[sl])
        w64 = np.exp(lw64.cpu().numpy()[sl])
        inr32, inr64 = (j32 >= 0) & (j32 < 400), (j64 >= 0) & (j64 < 400)
        same = (j32 == j64) & inr32
        d1 = np.bincount(j32[inr32], w32[inr32], 400) - np.bincount(j64[inr64], w64[inr64], 400)
        d2 = (np.bincount(j32[same], (w32[same] - w64[same]) ** 2, 400)
              + np.bincount(j32[inr32 & ~same], w32[inr32 & ~same] ** 2, 400)
              + np.bincount(j64[inr64 & ~same], w64[inr64 & ~same] ** 2, 400))
        sep = np.sqrt(np.maximum(d2 / n - (d1 / n) ** 2, 0.0) / n)
        ok = use & (sep > 0)
        zp = (d1[ok] / n) / sep[ok]
        allowed = int(binom.ppf(0.999, ok.sum(), 0.0027))
        paired.append((float(np.abs(zp).max()), int(np.sum(np.abs(zp) > 3)), allowed,
                       float(np.median(sep[ok] / (np.hypot(e1[ok], e2[ok]) * 0.0075)))))
        assert np.sum(np.abs(zp) > 3) <= allowed and np.abs(zp).max() < 5, (s, paired[-1])
    print("max |P32 - P64| / combined sigma per set:", [round(w, 3) for w in worst])
    print("paired: (max |z|, bins beyond 3, allowed, paired / combined sigma) per set:", paired)


def test_learned_bias_inference_full_size(nat):
    """The learned-bias stepper at its measured size: 2^26 runs of m = 1,
    phi_in = 8, wall at 9, dN = 5e-4, N_max = 60, k_eval = 64, with the
    benchmark's starting network (random hidden layers, output bias 0.4).
    E[w] = 1; the weighted P(N > 40) agrees with the survival PDE (1.0986e-3)
    within 4 standard errors + 0.5 %; runs sampled over the id range follow
    the oracle running the same BF16 network in binary64 (the paths differ
    only through the BF16 evaluation of b, so the medians of the per-run
    differences are small; a few runs drift apart); and the weighted P(N)
    agrees with 2^15 oracle runs of the same network bin by bin."""
    import torch
    norm = (5.2, 0.5, 30.0, 1.0 / 15.0)
    params = W.mlp_params(seed=5, gain=1.0, out_scale=0.05)
    params[-1] = 0.4
    w = nat.mlp_pack(params, norm)
    n, seed = 1 << 26, 12345
    spec = W.SetSpec(phi_in=8.0, m=1.0, b=0.0, dN=5e-4, n_max=60.0, n_traj=n, phi_uv=9.0)
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=60.0, mlp=w, k_eval=64)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    nat.fpt_simulate_mlp(p, nat.make_sets([spec]), seed, N, lw)
    x = torch.exp(lw)
    mw, sw = x.mean().item(), x.std().item() / math.sqrt(n)
    t = torch.where(N > 40.0, x, torch.zeros_like(x))
    P, sP = t.mean().item(), t.std().item() / math.sqrt(n)
    print(f"E[w] = {mw:.6f} +- {sw:.1e}; P(N > 40) = {P:.6e} +- {sP:.1e} (PDE 1.0986e-3)")
    assert abs(mw - 1) < 4 * sw
    assert abs(P - 1.0986e-3) < 4 * sP + 5e-3 * 1.0986e-3
    ids = _sample_ids(n, 96, 14)
    p64 = nat.mlp_unpack_bf16(params).numpy()

    def one(i):
        r = oracle.make_run(m=1.0, phi_in=8.0, phi_uv=9.0, dN=5e-4, n_max=60.0, seed=seed, traj_offset=int(i),
                            mlp=p64, mlp_norm=norm, k_eval=64)
        No, lo, _ = oracle.simulate(r, 1)
        return No[0], lo[0]
    with ThreadPoolExecutor(16) as ex:
        out = list(ex.map(one, ids))
    oN = np.array([o[0] for o in out])
    olw = np.array([o[1] for o in out])
    gN = N.cpu().numpy()[ids]
    glw = lw.cpu().numpy()[ids]
    fin = np.isfinite(gN) & np.isfinite(oN)
    dn = np.abs(gN[fin] - oN[fin])
    dl = np.abs(glw - olw)
    print(f"{ids.size} sampled runs: censoring agrees {np.mean(np.isinf(gN) == np.isinf(oN)):.3f}; |dN| median "
          f"{np.median(dn):.2e}, 90 % {np.quantile(dn, 0.9):.2e}; |d ln w| median {np.median(dl):.2e}, 90 % "
          f"{np.quantile(dl, 0.9):.2e}")
    assert np.mean(np.isinf(gN) == np.isinf(oN)) >= 0.95
    assert np.median(dn) < 5e-3 and np.median(dl) < 0.05
    # the weighted P(N) bin by bin (width 1 on (0, 60]) against 2^15 oracle runs of the same network
    m_o, chunk = 1 << 15, 1 << 11

    def part(k):
        r = oracle.make_run(m=1.0, phi_in=8.0, phi_uv=9.0, dN=5e-4, n_max=60.0, seed=seed + 1, traj_offset=k * chunk,
                            mlp=p64, mlp_norm=norm, k_eval=64)
        return oracle.simulate(r, chunk)[:2]
    with ThreadPoolExecutor(16) as ex:
        res = list(ex.map(part, range(m_o // chunk)))
    z = per_bin_z(N.cpu().numpy(), lw.cpu().numpy(), np.concatenate([a for a, _ in res]),
                  np.concatenate([b for _, b in res]), np.arange(0.0, 61.0, 1.0))
    assert_bins_agree(z, "learned bias at 2^26 runs vs 2^15 oracle runs")
