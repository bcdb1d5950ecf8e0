"""FP64 oracle of the per-bin estimators of arXiv:2206.11234, computed from the
raw records (first-passage time N_i, log-weight ln w_i) of every run.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: it shares no code with
the CUDA path, which works from the histogram's per-bin sums instead.

Per bin j = (lo + j d, lo + (j+1) d] (right-closed, §2.1 Eq. (9)):
  * direct / weighted naive estimate (§2.1 Eq. (9), §2.2 Eq. (16)):
        P_j = sum_{i in j} w_i / (d n_total),
    with standard error sqrt((sum w^2 / n_total - (sum w / n_total)^2) / n_total) / d;
  * lognormal estimate (§2.4 Eqs. (22)-(24)): with mu and s^2 the sample mean and
    the unbiased sample variance of ln w in the bin,
        <w> = exp(mu + s^2 / 2),  P_j = n_j <w> / (d n_total),
        eps_hi/lo = P_j |exp(+-a) - 1|,  a = sqrt(s^2 / n_j + s^4 / (2 n_j - 2));
  * normality of ln w in the bin (§2.4: D'Agostino and Pearson's omnibus test):
    K^2 = Z1(sqrt(b1))^2 + Z2(b2)^2 and p = exp(-K^2 / 2) (chi^2, 2 dof), with
    the skewness transform of D'Agostino (1970) and the kurtosis transform of
    Anscombe and Glynn (1983), as combined by D'Agostino, Belanger and
    D'Agostino (1990);
  * the lognormal estimate's next terms (reading of §2.4 Eq. (22)): ln <w> =
    k1 + k2/2 + k3/6 + k4/24 + ... in the cumulants of ln w; Eq. (22) keeps the
    first two, so bias_ln = k3/6 + k4/24 with the unbiased k-statistics k3, k4
    of ln w in the bin, and bias_se its standard error under normality,
    sqrt(var(k3)/36 + var(k4)/576), var(k3) = 6 n k2^3 / ((n-1)(n-2)),
    var(k4) = 24 n (n+1) k2^4 / ((n-1)(n-2)(n-3)) (Fisher's k-statistics;
    needs n_j >= 4 and s^2 > 0, NaN otherwise);
  * jackknife (§2.1): run i belongs to subset (id_offset + i) mod n_sub; each
    subset's estimate uses its own n_total; the spread of the n_sub estimates
    (unbiased variance) scaled from n_total / n_sub runs to n_total by the
    1/sqrt(n) law: sigma = std_k(P_k) / sqrt(n_sub).

Conventions where the paper is silent: an empty bin has P = 0 for both
estimators and eps = 0; the lognormal estimate needs n_j >= 2 (NaN otherwise);
the normality test needs n_j >= 8 and s^2 > 0 (NaN otherwise); the jackknife
needs n_sub >= 2 and every subset's estimate defined (NaN otherwise).

Parity status: pinned (tests/test_oracle_estimate.py) by scipy.stats.normaltest,
skewtest and kurtosistest on the same samples; the k-statistics by
scipy.stats.kstat and their variances by simulation of normal samples; the
bias terms by ln w with a gamma-shaped skew, whose <w> is known in closed form; by the lognormal mean and the
coverage of eps on exactly lognormal weights; by the reduction of Eq. (16) and
Eq. (23) to Eq. (9) when w = 1; by a hand-computed jackknife example.
"""
import math

import numpy as np

FIELDS = ("count", "p_direct", "se_direct", "p_lognormal", "eps_lo", "eps_hi", "mean_lw", "var_lw",
          "skew", "kurt", "z_skew", "z_kurt", "k2", "p_normal", "jk_direct", "jk_lognormal", "bias_ln", "bias_se")


def bin_index(N, n_bins, lo, hi):
    """Bin of every record (-1: N <= lo, N > hi or not finite), §2.1 Eq. (9)."""
    N = np.asarray(N, dtype=np.float64)
    d = (hi - lo) / n_bins
    j = np.full(N.shape, -1, dtype=np.int64)
    ok = np.isfinite(N) & (N > lo) & (N <= hi)
    jj = np.ceil((N[ok] - lo) / d).astype(np.int64) - 1
    j[ok] = np.clip(jj, 0, n_bins - 1)
    return j


def skewtest_z(x):
    """D'Agostino (1970): normal deviate of the sample skewness sqrt(b1)."""
    n = x.size
    c = x - x.mean()
    m2 = np.mean(c ** 2)
    m3 = np.mean(c ** 3)
    g = m3 / m2 ** 1.5
    y = g * math.sqrt((n + 1.0) * (n + 3.0) / (6.0 * (n - 2.0)))
    beta2 = (3.0 * (n * n + 27.0 * n - 70.0) * (n + 1.0) * (n + 3.0)
             / ((n - 2.0) * (n + 5.0) * (n + 7.0) * (n + 9.0)))
    w2 = -1.0 + math.sqrt(2.0 * (beta2 - 1.0))
    delta = 1.0 / math.sqrt(0.5 * math.log(w2))
    alpha = math.sqrt(2.0 / (w2 - 1.0))
    r = y / alpha
    return g, delta * math.log(r + math.sqrt(r * r + 1.0))


def kurtosistest_z(x):
    """Anscombe and Glynn (1983): normal deviate of the sample kurtosis b2."""
    n = x.size
    c = x - x.mean()
    m2 = np.mean(c ** 2)
    m4 = np.mean(c ** 4)
    b2 = m4 / (m2 * m2)
    mean = 3.0 * (n - 1.0) / (n + 1.0)
    var = 24.0 * n * (n - 2.0) * (n - 3.0) / ((n + 1.0) ** 2 * (n + 3.0) * (n + 5.0))
    z = (b2 - mean) / math.sqrt(var)
    sqrt_beta1 = (6.0 * (n * n - 5.0 * n + 2.0) / ((n + 7.0) * (n + 9.0))
                  * math.sqrt(6.0 * (n + 3.0) * (n + 5.0) / (n * (n - 2.0) * (n - 3.0))))
    A = 6.0 + 8.0 / sqrt_beta1 * (2.0 / sqrt_beta1 + math.sqrt(1.0 + 4.0 / sqrt_beta1 ** 2))
    t = (1.0 - 2.0 / A) / (1.0 + z * math.sqrt(2.0 / (A - 4.0)))
    cube = math.copysign(abs(t) ** (1.0 / 3.0), t)
    return b2, ((1.0 - 2.0 / (9.0 * A)) - cube) / math.sqrt(2.0 / (9.0 * A))


def dagostino_pearson(x):
    """(sqrt(b1), b2, Z1, Z2, K^2, p) of a sample (n >= 8, nonzero variance)."""
    x = np.asarray(x, dtype=np.float64)
    g, z1 = skewtest_z(x)
    b2, z2 = kurtosistest_z(x)
    k2 = z1 * z1 + z2 * z2
    return g, b2, z1, z2, k2, math.exp(-0.5 * k2)


def _direct(lw, n_total, d):
    if lw.size == 0:
        return 0.0, 0.0
    mx = lw.max()
    s1 = np.sum(np.exp(lw - mx))
    s2 = np.sum(np.exp(2.0 * (lw - mx)))
    p = math.exp(mx) * s1 / (n_total * d)
    v = s2 / n_total - (s1 / n_total) ** 2  # in units of exp(2 mx)
    return p, math.exp(mx) * math.sqrt(max(v, 0.0) / n_total) / d


def _lognormal(lw, n_total, d):
    n = lw.size
    if n == 0:
        return 0.0, 0.0, 0.0, math.nan, math.nan
    if n < 2:
        return math.nan, math.nan, math.nan, float(lw.mean()), math.nan
    mu = float(lw.mean())
    s2 = float(np.var(lw, ddof=1))
    p = n * math.exp(mu + 0.5 * s2) / (n_total * d)
    a = math.sqrt(s2 / n + s2 * s2 / (2.0 * n - 2.0))
    return p, p * (1.0 - math.exp(-a)), p * (math.exp(a) - 1.0), mu, s2


def subset_totals(n, n_sub, id_offset):
    """Number of runs of each jackknife subset among ids id_offset .. id_offset + n - 1."""
    k = (id_offset + np.arange(n, dtype=np.uint64)) % np.uint64(n_sub)
    return np.bincount(k.astype(np.int64), minlength=n_sub)


def lognormal_bias(x):
    """(k3/6 + k4/24, its standard error) from the unbiased k-statistics of the
    sample x (NaN for fewer than 4 values or zero variance)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4:
        return math.nan, math.nan
    c = x - x.mean()
    m2, m3, m4 = np.mean(c ** 2), np.mean(c ** 3), np.mean(c ** 4)
    if not m2 > 0:
        return math.nan, math.nan
    k2 = n / (n - 1) * m2
    k3 = n * n / ((n - 1) * (n - 2)) * m3
    k4 = n * n * ((n + 1) * m4 - 3 * (n - 1) * m2 * m2) / ((n - 1) * (n - 2) * (n - 3))
    v3 = 6 * n * k2 ** 3 / ((n - 1) * (n - 2))
    v4 = 24 * n * (n + 1) * k2 ** 4 / ((n - 1) * (n - 2) * (n - 3))
    return k3 / 6 + k4 / 24, math.sqrt(v3 / 36 + v4 / 576)


def estimate(N, logw, n_bins, lo, hi, n_sub=1, id_offset=0):
    """Per-bin estimators of the records (N_i, ln w_i), i = 0 .. n-1 (run ids
    id_offset + i).  Returns a dict of float64 arrays [n_bins], keys FIELDS."""
    N = np.asarray(N, dtype=np.float64)
    lw = np.asarray(logw, dtype=np.float64)
    n = N.size
    d = (hi - lo) / n_bins
    j = bin_index(N, n_bins, lo, hi)
    sub = ((id_offset + np.arange(n, dtype=np.uint64)) % np.uint64(n_sub)).astype(np.int64)
    tot_k = subset_totals(n, n_sub, id_offset)
    out = {f: np.full(n_bins, math.nan) for f in FIELDS}
    order = np.argsort(j, kind="stable")
    js = j[order]
    starts = np.searchsorted(js, np.arange(n_bins))
    ends = np.searchsorted(js, np.arange(n_bins), side="right")
    for b in range(n_bins):
        idx = order[starts[b]:ends[b]]
        x = lw[idx]
        out["count"][b] = x.size
        out["p_direct"][b], out["se_direct"][b] = _direct(x, n, d)
        (out["p_lognormal"][b], out["eps_lo"][b], out["eps_hi"][b],
         out["mean_lw"][b], out["var_lw"][b]) = _lognormal(x, n, d)
        out["bias_ln"][b], out["bias_se"][b] = lognormal_bias(x)
        if x.size >= 8 and out["var_lw"][b] > 0.0:
            (out["skew"][b], out["kurt"][b], out["z_skew"][b], out["z_kurt"][b],
             out["k2"][b], out["p_normal"][b]) = dagostino_pearson(x)
        if n_sub >= 2:
            pd = np.empty(n_sub)
            pl = np.empty(n_sub)
            for k in range(n_sub):
                xk = x[sub[idx] == k]
                pd[k] = _direct(xk, tot_k[k], d)[0] if tot_k[k] > 0 else math.nan
                pl[k] = _lognormal(xk, tot_k[k], d)[0] if tot_k[k] > 0 else math.nan
            out["jk_direct"][b] = np.std(pd, ddof=1) / math.sqrt(n_sub)
            out["jk_lognormal"][b] = np.std(pl, ddof=1) / math.sqrt(n_sub)
    return out


def pearson(N, logw):
    """Pearson's r of (N, ln w) over the runs with finite N (§3.4), with the
    count, means and unbiased (co)variances; r is NaN for fewer than 2 runs or
    a zero variance."""
    N = np.asarray(N, dtype=np.float64)
    lw = np.asarray(logw, dtype=np.float64)
    ok = np.isfinite(N)
    x, y = N[ok], lw[ok]
    n = x.size
    out = {"r": math.nan, "count": float(n), "mean_N": math.nan, "mean_lw": math.nan, "var_N": math.nan,
           "var_lw": math.nan, "cov": math.nan}
    if n >= 1:
        out["mean_N"], out["mean_lw"] = float(x.mean()), float(y.mean())
    if n >= 2:
        dx, dy = x - x.mean(), y - y.mean()
        sxx, syy, sxy = float(np.sum(dx * dx)), float(np.sum(dy * dy)), float(np.sum(dx * dy))
        out["var_N"], out["var_lw"], out["cov"] = sxx / (n - 1), syy / (n - 1), sxy / (n - 1)
        if sxx > 0 and syy > 0:
            out["r"] = sxy / math.sqrt(sxx * syy)
    return out


def stitch(estimates, estimator="lognormal", min_count=400, p_threshold=0.005):
    """Multi-bias reconstruction (§3.2): estimates = [estimate(...) of each
    simulation over the same bins].  Per bin, a simulation contributes if its
    bin holds >= min_count runs, its estimate is defined and > 0 and (lognormal)
    its normality p-value >= p_threshold (0: no test); the contributions are
    combined in log space with inverse-variance weights 1/a_k^2, a_k the
    relative error (lognormal: sqrt(s^2/n + s^4/(2n - 2) + 1/n), Eq. (24)'s
    spread of ln w plus the relative fluctuation of the count, which Eq. (24)
    leaves out and which is all that remains when w = 1; direct: se/p).  Returns {p, eps_lo, eps_hi, log_err, n_used, best} arrays."""
    n_bins = len(estimates[0]["count"])
    out = {f: np.full(n_bins, math.nan) for f in ("p", "eps_lo", "eps_hi", "log_err", "n_used", "best")}
    for j in range(n_bins):
        w, lp, aa, ks = [], [], [], []
        for k, e in enumerate(estimates):
            n = e["count"][j]
            if not n >= min_count:
                continue
            if estimator == "lognormal":
                if p_threshold > 0 and not e["p_normal"][j] >= p_threshold and not e["var_lw"][j] == 0:
                    continue  # zero variance (w = 1): a degenerate normal, kept
                p = e["p_lognormal"][j]
                s2 = e["var_lw"][j]
                a = math.sqrt(s2 / n + s2 * s2 / (2 * n - 2) + 1.0 / n)
            else:
                p = e["p_direct"][j]
                a = e["se_direct"][j] / p if p > 0 else math.nan
            if not (p > 0 and a > 0 and math.isfinite(p) and math.isfinite(a)):
                continue
            w.append(1.0 / (a * a))
            lp.append(math.log(p))
            aa.append(a)
            ks.append(k)
        out["n_used"][j] = len(w)
        out["best"][j] = -1
        if w:
            W = sum(w)
            a = 1.0 / math.sqrt(W)
            p = math.exp(sum(wi * li for wi, li in zip(w, lp)) / W)
            out["p"][j], out["log_err"][j] = p, a
            out["eps_lo"][j], out["eps_hi"][j] = p * (1 - math.exp(-a)), p * (math.exp(a) - 1)
            out["best"][j] = ks[int(np.argmin(aa))]
    return out
