"""GPU per-bin estimators (fpt_histogram -> fpt_estimate, from per-bin sums)
against the oracle's estimators computed from the raw records (§2.1 Eq. (9),
§2.2 Eq. (16), §2.4 Eqs. (22)-(24), the D'Agostino-Pearson test of §2.4, the
jackknife of §2.1).

Tolerances: both sides are binary64.  The GPU forms central moments from
moments about the bin maximum after merging subsets; the oracle centres the
samples first.  The re-centring amplifies rounding by at most (spread / sd)^k
for the k-th moment (spread = max - mean, a few sd here), so quantities built
from the first two moments agree to ~1e-12 and skewness / kurtosis statistics
to ~1e-9; the tests allow 1e-9 and 1e-7 respectively.  A wrong subset total,
a dropped re-centring term or a transposed moment index shows up at O(1).
"""
import math

import numpy as np
import pytest

from oracle import estimate as OE
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = ("p_direct", "se_direct", "p_lognormal", "eps_lo", "eps_hi", "mean_lw", "var_lw", "jk_direct",
         "jk_lognormal")
STATS = ("skew", "kurt", "z_skew", "z_kurt", "k2")


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _gpu_estimate(nat, N, lw, n_bins, lo, hi, n_sub=1, id_offset=0):
    import torch
    tN = torch.from_numpy(np.ascontiguousarray(N, dtype=np.float64)).cuda()
    tl = torch.from_numpy(np.ascontiguousarray(lw, dtype=np.float64)).cuda()
    bins = nat.empty_bins(n_bins * n_sub)
    counts = nat.empty_counts(1)
    nat.fpt_histogram(tN, tl, n_bins, lo, hi, bins, counts, n_sub=n_sub, id_offset=id_offset)
    est = nat.empty_estimates(n_bins)
    nat.fpt_estimate(bins, n_bins, lo, hi, len(N), est, n_sub=n_sub, id_offset=id_offset)
    return nat.estimates_to_dict(est)


def _compare(got, ref):
    np.testing.assert_array_equal(got["count"], ref["count"])
    for f in ref:
        assert np.array_equal(np.isnan(got[f]), np.isnan(ref[f])), f
    for f in TIGHT:
        np.testing.assert_allclose(got[f], ref[f], rtol=1e-9, atol=1e-300, equal_nan=True, err_msg=f)
    for f in STATS:
        np.testing.assert_allclose(got[f], ref[f], rtol=1e-7, atol=1e-7, equal_nan=True, err_msg=f)
    # k4 cancels between (n + 1) m4 and 3 (n - 1) m2^2 when ln w is near normal: the
    # bias terms are compared against their own statistical error
    np.testing.assert_allclose(got["bias_se"], ref["bias_se"], rtol=1e-7, equal_nan=True, err_msg="bias_se")
    ok = np.isfinite(ref["bias_ln"])
    assert np.all(np.abs(got["bias_ln"][ok] - ref["bias_ln"][ok]) <= 1e-6 * ref["bias_se"][ok] + 1e-12), "bias_ln"
    ok = np.isfinite(ref["p_normal"]) & (ref["p_normal"] > 1e-200)
    np.testing.assert_allclose(got["p_normal"][ok], ref["p_normal"][ok], rtol=1e-5)


def _drift_like_records(n, seed, lo, hi):
    """ln w correlated with N plus skewed noise, a few runs out of range or censored."""
    rng = np.random.default_rng(seed)
    N = rng.normal(0.5 * (lo + hi), 0.2 * (hi - lo), n)
    N[rng.random(n) < 0.01] = np.inf
    lw = -30.0 - 4.0 * (N - lo) + 0.8 * rng.standard_normal(n) + 0.3 * rng.exponential(1.0, n)
    lw[~np.isfinite(N)] = -1.0
    return N, lw


@pytest.mark.parametrize("n,n_bins,n_sub,id_offset", [(1, 5, 1, 0), (50, 4, 3, 7), (20000, 40, 1, 0),
                                                      (100003, 100, 16, 5), (300000, 256, 12, 123456789)])
def test_estimates_match_oracle(nat, n, n_bins, n_sub, id_offset):
    N, lw = _drift_like_records(n, seed=n, lo=7.0, hi=10.0)
    got = _gpu_estimate(nat, N, lw, n_bins, 7.0, 10.0, n_sub, id_offset)
    ref = OE.estimate(N, lw, n_bins, 7.0, 10.0, n_sub=n_sub, id_offset=id_offset)
    _compare(got, ref)


def test_estimates_wide_log_weights_and_unit_weights(nat):
    # ln w spread over tens of e-folds inside a bin (random_records), and w = 1
    N, lw = W.random_records(150000, seed=9, lo=0.0, hi=6.0)
    _compare(_gpu_estimate(nat, N, lw, 60, 0.0, 6.0, 10, 3), OE.estimate(N, lw, 60, 0.0, 6.0, n_sub=10, id_offset=3))
    z = np.zeros_like(lw)
    got = _gpu_estimate(nat, N, z, 60, 0.0, 6.0)
    _compare(got, OE.estimate(N, z, 60, 0.0, 6.0))
    ok = got["count"] >= 2
    np.testing.assert_array_equal(got["p_lognormal"][ok], got["p_direct"][ok])


def test_estimate_rejects_bad_arguments(nat):
    bins = nat.empty_bins(8)
    est = nat.empty_estimates(8)
    for args in ((0, 0.0, 1.0, 10, 1), (8, 1.0, 0.0, 10, 1), (8, 0.0, 1.0, 0, 1), (8, 0.0, 1.0, 10, 0),
                 (1024, 0.0, 1.0, 10, 5)):
        with pytest.raises(nat.FptError) as ei:
            nat.fpt_estimate(bins, args[0], args[1], args[2], args[3], est if args[0] <= 8 else
                             nat.empty_estimates(args[0]), n_sub=args[4])
        assert ei.value.code == nat.FPT_EINVAL


def test_lognormal_rule_on_simulated_runs(nat):
    """The §2.4 workflow on the GPU path: drift-dominated runs (m = 0.01, b = 1)
    have lognormal weights within a bin, and there the lognormal and the
    direct estimates agree within their errors; diffusion-dominated runs
    (m = 1, wall at 9, b = 0.4) fail the normality test by far."""
    import torch
    spec = W.SetSpec(phi_in=6.0, m=0.01, b=1.0, dN=1e-3, n_max=10.0, n_traj=1 << 20, hist_lo=8.45,
                     hist_hi=8.75, n_bins=30)
    wl = W.Workload("drift b=1", [spec], "f32_f64acc", seed=4)
    N, lw, _, _ = nat.simulate_workload(wl, with_hist=False)
    got = _gpu_estimate(nat, N.cpu().numpy(), lw.cpu().numpy(), spec.n_bins, spec.hist_lo, spec.hist_hi, 16, 0)
    big = got["count"] >= 400
    assert big.sum() >= 10
    p = got["p_normal"][big]
    assert np.median(p) > 0.05 and np.mean(p < 0.005) <= 0.1, p
    # the rule over the kept bins accepts the lognormal estimate here, while a
    # bin of a few dozen runs alone can refuse it
    assert nat.lognormal_applies(got)
    d = np.abs(got["p_lognormal"][big] - got["p_direct"][big])
    err = np.hypot(np.maximum(got["eps_lo"][big], got["eps_hi"][big]), got["se_direct"][big])
    assert np.mean(d <= 3 * err) >= 0.9
    spec = W.SetSpec(phi_in=8.0, m=1.0, b=0.4, dN=5e-4, n_max=60.0, phi_uv=9.0, n_traj=1 << 20, hist_lo=0.0,
                     hist_hi=60.0, n_bins=60)
    wl = W.Workload("diffusion b=0.4", [spec], "f32_f64acc", seed=4)
    N, lw, _, _ = nat.simulate_workload(wl, with_hist=False)
    got = _gpu_estimate(nat, N.cpu().numpy(), lw.cpu().numpy(), spec.n_bins, spec.hist_lo, spec.hist_hi)
    big = got["count"] >= 400
    assert big.sum() >= 20
    assert np.median(got["p_normal"][big]) < 1e-10
    assert not nat.lognormal_applies(got)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 1 << 20])
def test_pearson_matches_oracle(nat, n):
    import torch
    rng = np.random.default_rng(n + 3)
    N = rng.normal(8.5, 0.02, n)
    lw = -2.0 * (N - 8.5) / 0.02 + rng.normal(0, 0.5, n) - 40.0
    if n > 10:
        N[rng.random(n) < 0.01] = np.inf
    got = nat.fpt_pearson(torch.from_numpy(N).cuda(), torch.from_numpy(lw).cuda())
    ref = OE.pearson(N, lw)
    assert got["count"] == ref["count"]
    for f in ("r", "mean_N", "mean_lw", "var_N", "var_lw", "cov"):
        if math.isnan(ref[f]):
            assert math.isnan(got[f]), f
        else:
            assert math.isclose(got[f], ref[f], rel_tol=1e-10, abs_tol=1e-300), (f, got[f], ref[f])


def test_stitch_matches_oracle(nat):
    """Several record sets over the same bins (shifted, with their own weight
    spreads) through fpt_histogram -> fpt_estimate -> fpt_stitch against the
    oracle's estimate -> stitch on the same records."""
    import torch
    sets = []
    for k, (shift, spread) in enumerate(((0.0, 0.6), (0.8, 0.8), (1.6, 1.1))):
        rng = np.random.default_rng(40 + k)
        n = 200000
        N = rng.normal(8.5 + shift, 0.6, n)
        lw = -3.0 * shift - 2.0 * (N - 8.5 - shift) + spread * rng.standard_normal(n)
        sets.append((N, lw))
    nb, lo, hi = 60, 7.0, 12.0
    est = torch.stack([torch.from_numpy(np.stack([_gpu_estimate(nat, N, lw, nb, lo, hi)[f] for f in nat.ESTIMATE_FIELDS],
                                                 axis=1)) for N, lw in sets]).cuda()
    refs = [OE.estimate(N, lw, nb, lo, hi) for N, lw in sets]
    for kind, name in ((nat.ESTIMATOR_LOGNORMAL, "lognormal"), (nat.ESTIMATOR_DIRECT, "direct")):
        for pt in (0.0, 0.005):
            out = nat.fpt_stitch(est, estimator=kind, min_count=400, p_threshold=pt).cpu().numpy()
            ref = OE.stitch(refs, estimator=name, min_count=400, p_threshold=pt)
            np.testing.assert_array_equal(out[:, 4], ref["n_used"])
            np.testing.assert_array_equal(out[:, 5], ref["best"])
            for i, f in enumerate(("p", "eps_lo", "eps_hi", "log_err")):
                np.testing.assert_allclose(out[:, i], ref[f], rtol=1e-8, equal_nan=True, err_msg=f)
            assert (out[:, 4] >= 2).sum() >= 10  # the sets overlap
