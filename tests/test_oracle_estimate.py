"""Pins of the oracle's per-bin estimators (oracle/estimate.py): the normality
test against scipy.stats on the same samples, the lognormal estimate and the
coverage of its error bars on exactly lognormal weights (§2.4 Eqs. (22)-(24)),
the reduction of the weighted estimates to the direct one when w = 1 (§2.2
Eq. (16) -> §2.1 Eq. (9)) with the binomial standard error, and the
jackknife of §2.1 on hand-computed examples.  CPU only."""
import math
import warnings

import numpy as np
import pytest

from oracle import estimate as E

stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("n", [8, 9, 20, 57, 500, 20000])
@pytest.mark.parametrize("dist", ["normal", "lognormal", "uniform", "student3", "exponential"])
def test_dagostino_pearson_matches_scipy(n, dist):
    rng = np.random.default_rng(n * 7 + len(dist))
    x = {"normal": lambda: rng.normal(-40.0, 0.7, n), "lognormal": lambda: rng.lognormal(0.0, 0.8, n),
         "uniform": lambda: rng.uniform(-1.0, 1.0, n), "student3": lambda: rng.standard_t(3, n),
         "exponential": lambda: rng.exponential(2.0, n)}[dist]()
    g, b2, z1, z2, k2, p = E.dagostino_pearson(x)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        zs = stats.skewtest(x).statistic
        zk = stats.kurtosistest(x).statistic
        nt = stats.normaltest(x)
    assert math.isclose(g, stats.skew(x), rel_tol=1e-9, abs_tol=1e-12)
    assert math.isclose(b2, stats.kurtosis(x, fisher=False), rel_tol=1e-9)
    assert math.isclose(z1, zs, rel_tol=1e-9, abs_tol=1e-10)
    assert math.isclose(z2, zk, rel_tol=1e-9, abs_tol=1e-10)
    assert math.isclose(k2, nt.statistic, rel_tol=1e-9, abs_tol=1e-10)
    assert math.isclose(p, nt.pvalue, rel_tol=1e-9, abs_tol=1e-300)


def test_lognormal_estimate_and_error_coverage():
    """ln w ~ Normal(mu, sigma^2) in one bin: <w> = exp(mu + sigma^2/2) (Eq. (22));
    the interval [P - eps_lo, P + eps_hi] (Eq. (24)) covers the truth about 68 %
    of the time.  Dropping the sigma^4 term would cover ~51 %."""
    mu, sig, n, reps = -3.0, 1.5, 60, 600
    truth = math.exp(mu + 0.5 * sig * sig)
    rng = np.random.default_rng(1)
    hit, est = 0, []
    for r in range(reps):
        lw = rng.normal(mu, sig, n)
        o = E.estimate(np.full(n, 0.5), lw, 1, 0.0, 1.0)
        p, lo, hi = o["p_lognormal"][0], o["eps_lo"][0], o["eps_hi"][0]
        hit += (p - lo <= truth <= p + hi)
        est.append(p)
        assert math.isclose(o["mean_lw"][0], lw.mean(), rel_tol=1e-12)
        assert math.isclose(o["var_lw"][0], lw.var(ddof=1), rel_tol=1e-12)
    cover = hit / reps
    assert 0.62 <= cover <= 0.74, cover
    assert abs(np.mean(est) / truth - 1) < 0.03


def test_unit_weights_reduce_to_direct_estimate():
    """w = 1 for every run (b = 0): Eq. (16) and Eq. (23) both give Eq. (9),
    n_j / (d n_total), with the binomial standard error."""
    rng = np.random.default_rng(2)
    n, nb, lo, hi = 5000, 25, 0.0, 5.0
    N = rng.gamma(3.0, 0.6, n)
    N[rng.random(n) < 0.03] = np.inf
    o = E.estimate(N, np.zeros(n), nb, lo, hi)
    d = (hi - lo) / nb
    edges = np.linspace(lo, hi, nb + 1)
    cnt = np.histogram(N[np.isfinite(N) & (N > lo) & (N <= hi)], bins=edges)[0]
    np.testing.assert_array_equal(o["count"], cnt)
    q = cnt / n
    np.testing.assert_allclose(o["p_direct"], q / d, rtol=1e-12)
    np.testing.assert_allclose(o["se_direct"], np.sqrt(q * (1 - q) / n) / d, rtol=1e-9, atol=1e-15)
    ok = cnt >= 2
    np.testing.assert_allclose(o["p_lognormal"][ok], q[ok] / d, rtol=1e-12)
    assert np.all(o["eps_lo"][ok] == 0) and np.all(o["eps_hi"][ok] == 0)
    assert np.all(np.isnan(o["p_normal"]))  # zero variance: the test is undefined


def test_jackknife_hand_examples():
    """Four runs in one bin (0, 1], weights 1, 2, 1, 4 (ids 0..3), two subsets
    by id parity: subset 0 = {1, 1} -> P0 = 2/2 = 1, subset 1 = {2, 4} -> P1 =
    6/2 = 3; the spread (unbiased) is sqrt(2), scaled by 1/sqrt(2): 1.  The
    full estimate is 8/4 = 2.  With ids 1..4 the subsets swap."""
    N = np.full(4, 0.5)
    lw = np.log([1.0, 2.0, 1.0, 4.0])
    o = E.estimate(N, lw, 1, 0.0, 1.0, n_sub=2)
    assert math.isclose(o["p_direct"][0], 2.0, rel_tol=1e-15)
    assert math.isclose(o["jk_direct"][0], 1.0, rel_tol=1e-14)
    o1 = E.estimate(N, lw, 1, 0.0, 1.0, n_sub=2, id_offset=1)
    assert math.isclose(o1["jk_direct"][0], 1.0, rel_tol=1e-14)
    # three subsets of 5 runs (ids 2..6 -> subsets 2, 0, 1, 2, 0): totals 2, 1, 2;
    # weights 3, 1, 2, 5, 1 -> P0 = (1 + 1)/2 = 1, P1 = 2/1 = 2, P2 = (3 + 5)/2 = 4;
    # mean 7/3, unbiased variance ((4/3)^2 + (1/3)^2 + (5/3)^2)/2 = 7/3, scaled by 1/sqrt(3)
    lw3 = np.log([3.0, 1.0, 2.0, 5.0, 1.0])
    o3 = E.estimate(np.full(5, 0.5), lw3, 1, 0.0, 1.0, n_sub=3, id_offset=2)
    assert math.isclose(o3["jk_direct"][0], math.sqrt(7.0 / 3.0) / math.sqrt(3.0), rel_tol=1e-14)
    np.testing.assert_array_equal(E.subset_totals(5, 3, 2), [2, 1, 2])


def test_jackknife_agrees_with_standard_error_statistically():
    """Direct sampling: the jackknife over 20 subsets and the analytic standard
    error estimate the same binomial spread (bins with >= 400 runs, §2.1)."""
    rng = np.random.default_rng(3)
    n = 200000
    N = rng.gamma(4.0, 0.5, n)
    o = E.estimate(N, np.zeros(n), 20, 0.0, 6.0, n_sub=20)
    ok = o["count"] >= 400
    r = o["jk_direct"][ok] / o["se_direct"][ok]
    assert ok.sum() >= 10
    assert 0.85 < np.median(r) < 1.15 and np.all((r > 0.4) & (r < 1.8))


def test_edge_cases():
    N = np.array([0.5, 1.5, 1.6, np.inf, -1.0])
    lw = np.array([-2.0, -1.0, -3.0, 0.0, 0.0])
    o = E.estimate(N, lw, 3, 0.0, 3.0, n_sub=2)
    assert o["count"].tolist() == [1, 2, 0]
    assert math.isnan(o["p_lognormal"][0])          # one run: no variance
    assert math.isclose(o["p_direct"][0], math.exp(-2.0) / 5.0)
    assert o["p_direct"][2] == 0 and o["p_lognormal"][2] == 0 and o["eps_hi"][2] == 0
    assert np.all(np.isnan(o["k2"]))                # fewer than 8 runs
    assert math.isnan(o["jk_lognormal"][1])         # subset 1 holds one run of bin 1


def test_pearson_matches_scipy_and_exact_cases():
    rng = np.random.default_rng(8)
    N = rng.normal(8.5, 0.02, 5000)
    lw = -3.0 * (N - 8.5) / 0.02 + rng.normal(0, 1.0, N.size)
    N[::97] = np.inf
    o = E.pearson(N, lw)
    ok = np.isfinite(N)
    assert math.isclose(o["r"], stats.pearsonr(N[ok], lw[ok]).statistic, rel_tol=1e-12)
    assert o["count"] == ok.sum()
    assert math.isclose(o["cov"], np.cov(N[ok], lw[ok])[0, 1], rel_tol=1e-12)
    # exactly linear: r = +-1; constant: undefined
    x = np.linspace(1.0, 2.0, 11)
    assert math.isclose(E.pearson(x, 3 * x - 1)["r"], 1.0, rel_tol=1e-14)
    assert math.isclose(E.pearson(x, -0.5 * x)["r"], -1.0, rel_tol=1e-14)
    assert math.isnan(E.pearson(x, np.zeros(11))["r"])
    assert math.isnan(E.pearson(np.array([np.inf, 1.0]), np.zeros(2))["r"])


def _fake_estimate(p, var, count, p_normal=0.5):
    n = len(p)
    e = {f: np.full(n, math.nan) for f in E.FIELDS}
    e["p_lognormal"], e["var_lw"], e["count"] = np.array(p, float), np.array(var, float), np.array(count, float)
    e["p_normal"] = np.full(n, p_normal)
    e["p_direct"] = np.array(p, float)
    e["se_direct"] = np.array(p, float) * 0.1
    return e


def test_stitch_hand_example_and_filters():
    """Two simulations of one bin: relative errors a1 = 0.1, a2 = 0.2 (set up
    through var and count with the count term included) -> weights 100 and 25,
    ln p = (100 ln 1e-10 + 25 ln 2e-10) / 125 -> p = 1e-10 * 2^0.2, a = 1/sqrt(125)."""
    n = 10000.0
    # choose var so that var/n + var^2/(2n - 2) + 1/n = a^2
    def var_for(a):
        c = 1.0 / (2 * n - 2)
        return (-1.0 / n + math.sqrt(1.0 / n ** 2 + 4 * c * (a * a - 1.0 / n))) / (2 * c)
    e1 = _fake_estimate([1e-10], [var_for(0.1)], [n])
    e2 = _fake_estimate([2e-10], [var_for(0.2)], [n])
    o = E.stitch([e1, e2])
    assert math.isclose(o["p"][0], 1e-10 * 2 ** 0.2, rel_tol=1e-12)
    assert math.isclose(o["log_err"][0], 1 / math.sqrt(125), rel_tol=1e-12)
    assert o["n_used"][0] == 2 and o["best"][0] == 0
    # a single simulation is returned as it is
    o1 = E.stitch([e1])
    assert math.isclose(o1["p"][0], 1e-10, rel_tol=1e-14) and math.isclose(o1["log_err"][0], 0.1, rel_tol=1e-12)
    # filters: too few runs, failed normality, nothing left
    assert E.stitch([_fake_estimate([1e-10], [0.5], [399])])["n_used"][0] == 0
    assert math.isnan(E.stitch([_fake_estimate([1e-10], [0.5], [1000], p_normal=0.001)])["p"][0])
    o2 = E.stitch([e1, _fake_estimate([5e-10], [0.5], [1000], p_normal=0.001)])
    assert o2["n_used"][0] == 1 and math.isclose(o2["p"][0], 1e-10, rel_tol=1e-14)
    # w = 1 in the bin: zero variance, no normality test, kept with the count's error 1/sqrt(n)
    o3 = E.stitch([_fake_estimate([3e-3], [0.0], [2500], p_normal=math.nan)])
    assert o3["n_used"][0] == 1 and math.isclose(o3["log_err"][0], 1 / 50, rel_tol=1e-12)
    od = E.stitch([e1, e2], estimator="direct")
    assert math.isclose(od["p"][0], math.sqrt(1e-10 * 2e-10), rel_tol=1e-12)  # equal relative errors


def test_stitch_error_covers_the_truth():
    """K simulations of the same lognormal bin: the combined estimate's interval
    covers the true mean about 68 % of the time."""
    rng = np.random.default_rng(5)
    mu, sig, reps = -5.0, 1.2, 300
    truth = math.exp(mu + sig * sig / 2)
    hit = 0
    for r in range(reps):
        ests = []
        for k in range(4):
            n = int(rng.integers(400, 2000))
            lw = rng.normal(mu, sig, n)
            ests.append(E.estimate(np.full(n, 0.5), lw, 1, 0.0, 1.0))
            # a bin holding all n runs of n_total = n: P = <w> exactly as Eq. (23) with n_j = n_total
        o = E.stitch(ests, p_threshold=0.0)
        hit += (o["p"][0] - o["eps_lo"][0] <= truth <= o["p"][0] + o["eps_hi"][0])
    assert 0.58 <= hit / reps <= 0.80, hit / reps


def test_bias_terms_match_kstat_and_their_spread():
    """bias_ln = k3/6 + k4/24 with scipy's unbiased k-statistics; bias_se is
    the spread of that quantity over normal samples (Fisher's variances)."""
    rng = np.random.default_rng(8)
    for n in (4, 9, 50, 3000):
        x = rng.gamma(3.0, 1.0, n) - 7.0
        b, se = E.lognormal_bias(x)
        assert math.isclose(b, stats.kstat(x, 3) / 6 + stats.kstat(x, 4) / 24, rel_tol=1e-9, abs_tol=1e-12)
        assert se > 0
    for n in (50, 200, 2000):
        sig = 2.5
        draws = [E.lognormal_bias(rng.normal(1.0, sig, n)) for _ in range(4000)]
        b = np.array([d[0] for d in draws])
        se = np.array([d[1] for d in draws])
        # the spread of the estimate is the standard error at the true variance;
        # the estimated standard error (through k2) approaches it as n grows
        v = sig ** 2
        true_se = math.sqrt(6 * n * v ** 3 / ((n - 1) * (n - 2)) / 36 + 24 * n * (n + 1) * v ** 4 / ((n - 1) * (n - 2) * (n - 3)) / 576)
        assert abs(b.std() / true_se - 1) < 0.06, (n, b.std(), true_se)
        assert abs(b.mean()) < 4 * b.std() / math.sqrt(b.size)
        if n >= 2000:
            assert abs(np.median(se) / true_se - 1) < 0.05
    assert all(math.isnan(v) for v in E.lognormal_bias([1.0, 2.0, 3.0]))
    assert all(math.isnan(v) for v in E.lognormal_bias([1.0] * 10))


@pytest.mark.parametrize("sigma2,skew,n", [(31.0, -3e-3, 100000), (31.0, 0.05, 100000), (4.0, 0.2, 20000)])
def test_bias_terms_correct_the_lognormal_estimate(sigma2, skew, n):
    """ln w = c + sign sigma (G - k)/sqrt(k), G ~ Gamma(k, 1): variance sigma^2,
    skewness sign 2/sqrt(k), and ln <w> = c - sign sigma sqrt(k) - k ln(1 - sign
    sigma / sqrt(k)) exactly.  Eq. (22)'s estimate misses ln <w> by about
    k3/6 + k4/24; adding bias_ln removes that within its error bias_se, over
    repeated bins, and the corrected interval covers the truth."""
    rng = np.random.default_rng(int(1e4 * abs(skew)) + int(sigma2))
    sig, sgn = math.sqrt(sigma2), math.copysign(1.0, skew)
    k = (2.0 / abs(skew)) ** 2
    c = -40.0
    x = sgn * sig / math.sqrt(k)
    truth = c - sgn * sig * math.sqrt(k) - k * math.log1p(-x)
    miss, dev, cover = [], [], 0
    reps = 40
    for r in range(reps):
        lw = c + sgn * sig * (rng.gamma(k, 1.0, n) - k) / math.sqrt(k)
        o = E.estimate(np.full(n, 0.5), lw, 1, 0.0, 1.0)
        ln_p = math.log(o["p_lognormal"][0])  # d = 1 and n_total = n_j: the estimate of <w>
        miss.append(ln_p - truth)
        d = ln_p + o["bias_ln"][0] - truth
        dev.append(d)
        a = math.sqrt(o["var_lw"][0] / n + o["var_lw"][0] ** 2 / (2 * n - 2))
        cover += abs(d) <= 2 * math.hypot(o["bias_se"][0], a)
    expected_miss = -(sgn * 2 * sig ** 3 / math.sqrt(k) / 6 + 6 * sig ** 4 / k / 24)  # -(k3/6 + k4/24)
    miss, dev = np.array(miss), np.array(dev)
    se = dev.std(ddof=1) / math.sqrt(reps)
    assert abs(miss.mean() - expected_miss) < 4 * miss.std(ddof=1) / math.sqrt(reps) + 0.05 * abs(expected_miss)
    assert abs(dev.mean()) < 4 * se, (dev.mean(), se, miss.mean())
    assert cover >= 0.85 * reps
