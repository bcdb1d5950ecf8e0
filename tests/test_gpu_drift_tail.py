"""The far tail of drift domination on the GPU path against the saddle-point
density of the exact generating function K(s) = ln E[e^{sN}] (tests/analytic.py:
the Riccati form of Appendix A's backward equation, pinned on the CPU against
closed forms, the hypergeometric solution and the backward cumulants).

Quadratic inflation, m = 0.01, phi_in = 6, dN = 1e-3 (§3.3 regime):
sigma_N = 0.0203, and the noise-free Euler-Maruyama map reaches phi_end
dN/2 ln(phi_in/phi_end) = 7.2e-4 later than the continuum, so the reference
density is taken at N minus that delay.

* Constant bias, the benchmark's ladder b = 0, 0.5, 1, 2, 4 x 2^22 runs
  (binary32 state, compensated binary32 log-weight): <N> of the unbiased set
  is K'(0) plus the delay within 4 standard errors (the delay is 70 of them);
  the lognormal estimates (Eq. (23)) of the sets whose ln w spreads little
  within a bin (b <= 1, variance <= 2) agree with the reference within 4
  errors + 1 % from 4 sigma below the mean to 7 sigma above it.
* Power-law bias p = 3 (§3.4 Eq. (26), |r| = 0.99996), amplitudes placing the
  classical sample duration 5.3 and 10.7 sigma past the target's, 2^22 runs
  each (binary32 state, binary64 log-weight): the direct estimates (Eq. (16))
  of every bin with >= 400 runs agree with the reference within 4 standard
  errors + 1 % out to 14.6 sigma (P ~ 1e-43).  The 1 % covers the O(dN)
  discretisation error left after the delay (+0.55 % at dN = 1e-3, +0.33 % at
  5e-4 in the mean over the tail bins).

* The paper's own drift-dominated workloads, binary64: §3.3 Fig. 9 (m = 0.001,
  wall at phi_in = sqrt(42)): <N> and the lognormal estimates of A <= 2, and
  at A = 3 (Fig. 1) the naive estimator's shortfall; §3.4 Fig. 10 (p = 3
  against p = 1 at 4e4 runs): the p = 3 naive estimates and their smaller
  errors.

For the b = 2 and b = 4 sets the lognormal estimates are printed, and the
cumulant-corrected ones asserted.  At b = 4 ln w has variance ~31 within a
bin; there Eq. (22)'s estimate lies about +0.10 in ln P above the reference
(weighted mean over its bins), outside Eq. (24)'s error, because a skewness of
ln w of a few 1e-3 (below what the normality test can see at these counts)
moves exp(mu + sigma^2/2) by that much.  Adding the bin's k3/6 + k4/24
(fpt_estimate's bias_ln, error bias_se) brings every bin within 5 of its
errors and the weighted mean over the bins within 4 pooled errors + 1 %.
"""
import math

import numpy as np
import pytest

import analytic as A
from paper_2206_11234_gb300 import power_bias as PB
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SQ2 = math.sqrt(2.0)
M, PHI_IN, DN = 0.01, 6.0, 1e-3
NB, LO, HI, N_SUB = 400, 7.0, 10.0, 10
EDGES = LO + (HI - LO) / NB * np.arange(NB + 1)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


@pytest.fixture(scope="module")
def reference():
    """Bin averages of the saddle-point density at N - delay, its cumulants and
    the delay (the wall at 7 is never felt: escape against the drift ~ e^-35000)."""
    D = lambda x: A.quad_drift(x, 0.0, M)
    S = lambda x: A.quad_noise(x, M)
    mgf = lambda s: A.mgf_cumulants(s, PHI_IN, D, S, SQ2, 7.0)
    sp = A.SaddlepointDensity.from_mgf(np.arange(-300.0, 901.0, 25.0), mgf)
    k = mgf(0.0)
    delay = A.em_classical_shift(PHI_IN, DN)
    lo_ok, hi_ok = float(sp.K1(sp.s[0])), float(sp.K1(sp.s[-1]))
    P = np.full(NB, np.nan)
    for j in range(NB):
        a, b = EDGES[j] - delay, EDGES[j + 1] - delay
        if a > lo_ok and b < hi_ok:
            P[j] = sp.bin_average(a, b)
    return P, k[1], math.sqrt(k[2]), delay


def _estimates(nat, N, lw, n):
    import torch
    bins = nat.empty_bins(NB * N_SUB)
    counts = nat.empty_counts(1)
    nat.fpt_histogram(N, lw, NB, LO, HI, bins, counts, n_sub=N_SUB)
    est = nat.empty_estimates(NB)
    nat.fpt_estimate(bins, NB, LO, HI, n, est, n_sub=N_SUB)
    torch.cuda.synchronize()
    return nat.estimates_to_dict(est)


def _z(mean, sig):
    return (0.5 * (EDGES[:-1] + EDGES[1:]) - mean) / sig


def test_constant_bias_ladder(nat, reference):
    P, k1, sig, delay = reference
    wl = W.drift_dominated_ladder()
    N, lw, _, _ = nat.simulate_workload(wl, with_hist=False)
    n = wl.sets[0].n_traj
    N0 = N[:n].cpu().numpy()
    se = N0.std() / math.sqrt(n)
    print(f"<N> - K'(0) = {N0.mean() - k1:.3e}, delay {delay:.3e}, se {se:.2e}")
    assert abs(N0.mean() - k1 - delay) < 4 * se
    assert delay > 50 * se
    z = _z(k1, sig)
    for k, s in enumerate(wl.sets):
        e = _estimates(nat, N[k * n:(k + 1) * n].contiguous(), lw[k * n:(k + 1) * n].contiguous(), n)
        use = (e["count"] >= 400) & np.isfinite(P) & (e["p_lognormal"] > 0)
        dev = np.log(e["p_lognormal"][use] / P[use])
        # Eq. (24)'s error plus the count's own fluctuation, which it leaves out
        # (all the error there is when w = 1)
        err = np.hypot(0.5 * (e["eps_lo"][use] + e["eps_hi"][use]) / e["p_lognormal"][use],
                       1 / np.sqrt(e["count"][use]))
        w = 1 / err ** 2
        print(f"b {s.b}: {use.sum()} bins, z {z[use].min():.1f}..{z[use].max():.1f}, P down to {P[use].min():.2e}, "
              f"weighted mean ln(p/P) {np.sum(w * dev) / np.sum(w):+.4f}, max |dev|/err {np.max(np.abs(dev) / err):.2f}, "
              f"median var ln w {np.median(e['var_lw'][use]):.3g}")
        if s.b <= 1.0:
            assert use.sum() >= 10
            assert np.all(np.abs(dev) <= 4 * err + 0.01), (s.b, np.max(np.abs(dev) / (4 * err + 0.01)))
            assert np.median(e["var_lw"][use]) <= 2.5
        if s.b >= 2.0:
            # the cumulant-corrected estimate p_lognormal exp(k3/6 + k4/24): its error per
            # bin is dominated by bias_se; pooled over the bins it removes the offset
            # that Eq. (22) leaves where ln w spreads widely (the bins are independent)
            ok = use & np.isfinite(e["bias_ln"])
            devc = dev[ok[use]] + e["bias_ln"][ok]
            errc = np.hypot(err[ok[use]], e["bias_se"][ok])
            wc = 1 / errc ** 2
            mc, sc = np.sum(wc * devc) / np.sum(wc), 1 / math.sqrt(np.sum(wc))
            mu = np.sum(wc * dev[ok[use]]) / np.sum(wc)
            print(f"b {s.b}: corrected weighted mean ln(p/P) {mc:+.4f} +- {sc:.4f} (uncorrected, same weights, "
                  f"{mu:+.4f}); max |dev|/err corrected {np.max(np.abs(devc) / errc):.2f}")
            assert ok.sum() >= 10
            assert abs(mc) <= 4 * sc + 0.01, (s.b, mc, sc)
            assert np.all(np.abs(devc) <= 5 * errc + 0.01), (s.b, np.max(np.abs(devc) / errc))


def test_power_law_bias_far_tail(nat, reference):
    import torch
    P, k1, sig, delay = reference
    sig_cl = PB.classical_sigma(M, PHI_IN)
    n_t = PB.classical_duration(0.0, 1.0, PHI_IN)
    n = 1 << 22
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    z = _z(k1, sig)
    deepest = 1.0
    for shift in (5.3, 10.7):
        amp = PB.tune_amplitude(3.0, n_t + shift * sig_cl, PHI_IN)
        prm = nat.make_params(precision="f32_f64acc", m=M, n_max=HI, bias_p=3.0)
        nat.fpt_simulate(prm, n, PHI_IN, SQ2, math.inf, DN, amp, 0, N, lw)
        r = nat.fpt_pearson(N, lw)
        e = _estimates(nat, N, lw, n)
        use = (e["count"] >= 400) & np.isfinite(P) & (e["p_direct"] > 0)
        dev = np.log(e["p_direct"][use] / P[use])
        rel = e["se_direct"][use] / e["p_direct"][use]
        w = 1 / rel ** 2
        devl = np.log(e["p_lognormal"][use] / P[use])
        print(f"p = 3, shift {shift} sigma: |r| {abs(r['r']):.6f}, {use.sum()} bins, z {z[use].min():.1f}.."
              f"{z[use].max():.1f}, P down to {P[use].min():.2e}; direct: weighted mean ln(p/P) "
              f"{np.sum(w * dev) / np.sum(w):+.4f}, max |dev|/se {np.max(np.abs(dev) / rel):.2f}; lognormal: "
              f"weighted mean {np.sum(w * devl) / np.sum(w):+.4f}, bins failing the normality test "
              f"{np.mean(e['p_normal'][use] < 0.005):.2f}")
        assert abs(r["r"]) > 0.9999
        assert use.sum() >= 15
        assert np.all(np.abs(dev) <= 4 * rel + 0.01), np.max(np.abs(dev) / (4 * rel + 0.01))
        deepest = min(deepest, P[use].min())
    assert deepest < 1e-40


def test_fig9_paper_workload(nat):
    """§3.3 Fig. 9: m = 0.001, phi_in = phi_uv = sqrt(42), A = 0 .. 4, 2^18 runs
    per amplitude (the paper uses 2e5), dN = sigma_N / 20 (the paper gives no
    dN), binary64 path, 100 bins of sigma_N / 4 from -6 to +19 sigma.  <N> is
    K'(0) plus the Euler-Maruyama delay; the lognormal estimates of A <= 2
    (variance of ln w in a bin <= 9) agree with the saddle point within 4
    errors + 1 %.  At A = 3 (the paper's Fig. 1) the naive estimates fall well
    below P (the sampling problem of §2.4) while the lognormal ones lie within
    0.1 in ln P.  A = 3 and 4 are printed (the lognormal estimator's bias
    grows with that variance: +4 % and +7 % there, P ~ 1e-41), with the
    Gaussian approximation the paper draws, which the skewness of N puts 0.6
    below the saddle point in ln P at 11 sigma and 1.1 below at 14 sigma."""
    import torch
    R42 = math.sqrt(42.0)
    m = 1e-3
    D = lambda x: A.quad_drift(x, 0.0, m)
    S = lambda x: A.quad_noise(x, m)
    mgf = lambda s: A.mgf_cumulants(s, R42, D, S, SQ2, R42)
    k = mgf(0.0)
    sig = math.sqrt(k[2])
    dN = sig / 20
    sp = A.SaddlepointDensity.from_mgf(np.arange(-2000.0, 8001.0, 200.0), mgf)
    delay = A.em_classical_shift(R42, dN)
    nb, lo, hi = 100, k[1] - 6 * sig, k[1] + 19 * sig
    edges = lo + (hi - lo) / nb * np.arange(nb + 1)
    P = np.array([sp.bin_average(edges[j] - delay, edges[j + 1] - delay)
                  if sp.K1(sp.s[0]) < edges[j] - delay and edges[j + 1] - delay < sp.K1(sp.s[-1]) else np.nan
                  for j in range(nb)])
    mid = 0.5 * (edges[1:] + edges[:-1]) - delay
    gauss = np.exp(-0.5 * ((mid - k[1]) / sig) ** 2) / math.sqrt(2 * math.pi * k[2])
    n, amps = 1 << 18, (0.0, 1.0, 2.0, 3.0, 4.0)
    specs = [W.SetSpec(phi_in=R42, m=m, b=a, dN=dN, n_max=hi, n_traj=n, phi_uv=R42, set_id=i, hist_lo=lo,
                       hist_hi=hi, n_bins=nb) for i, a in enumerate(amps)]
    N, lw, _, _ = nat.simulate_workload(W.Workload("fig9", specs, "f64", seed=0), with_hist=False)
    N0 = N[:n].cpu().numpy()
    se = N0.std() / math.sqrt(n)
    print(f"<N> - K'(0) = {N0.mean() - k[1]:.3e}, delay {delay:.3e}, se {se:.1e}; Var N / K''(0) {N0.var() / k[2]:.5f}")
    assert abs(N0.mean() - k[1] - delay) < 4 * se and delay > 15 * se
    z = (0.5 * (edges[1:] + edges[:-1]) - k[1]) / sig
    for i, a in enumerate(amps):
        bins = nat.empty_bins(nb * N_SUB)
        counts = nat.empty_counts(1)
        nat.fpt_histogram(N[i * n:(i + 1) * n].contiguous(), lw[i * n:(i + 1) * n].contiguous(), nb, lo, hi, bins,
                          counts, n_sub=N_SUB)
        est = nat.empty_estimates(nb)
        nat.fpt_estimate(bins, nb, lo, hi, n, est, n_sub=N_SUB)
        torch.cuda.synchronize()
        e = nat.estimates_to_dict(est)
        use = (e["count"] >= 400) & np.isfinite(P)
        dev = np.log(e["p_lognormal"][use] / P[use])
        err = np.hypot(0.5 * (e["eps_lo"][use] + e["eps_hi"][use]) / e["p_lognormal"][use],
                       1 / np.sqrt(e["count"][use]))
        w = 1 / err ** 2
        print(f"A {a}: z {z[use].min():.1f}..{z[use].max():.1f}, P down to {P[use].min():.1e}, lognormal weighted "
              f"mean ln(p/P) {np.sum(w * dev) / np.sum(w):+.4f}, max |dev|/err {np.max(np.abs(dev) / err):.2f}, "
              f"median var ln w {np.median(e['var_lw'][use]):.3g}; ln(Gaussian/P) at the deepest bin "
              f"{math.log(gauss[use][-1] / P[use][-1]):+.3f}")
        devd = np.log(np.maximum(e["p_direct"][use], 1e-300) / P[use])
        wd = e["count"][use]
        print(f"      direct (Eq. (16)) count-weighted mean ln(p/P) {np.sum(wd * devd) / np.sum(wd):+.3f}")
        assert use.sum() >= 15
        if a <= 2.0:
            assert np.all(np.abs(dev) <= 4 * err + 0.01), (a, np.max(np.abs(dev) / (4 * err + 0.01)))
        if a == 3.0:
            # Fig. 1 (same m, phi_in and A): the naive estimate misses the rare
            # large weights and falls well below P, the lognormal one does not
            assert np.sum(wd * devd) / np.sum(wd) < -0.5
            assert abs(np.sum(w * dev) / np.sum(w)) < 0.1


def test_fig10_power_law_against_constant_bias(nat):
    """§3.4 Fig. 10: m = 0.001, phi_in = 6 (the paper does not give it), no
    wall, A_p placing the classical sample duration 8 sigma past the target's,
    4e4 runs per p (the paper's count), dN = sigma_N / 20, binary64 path.  The
    naive estimates of the p = 3 set agree with the saddle point within 4
    standard errors + 1 % in every bin with >= 400 runs, with smaller errors
    than the lognormal estimates of the p = 1 set in the same bins (printed
    against the reference too)."""
    import torch
    m, phi_in = 1e-3, 6.0
    D = lambda x: A.quad_drift(x, 0.0, m)
    S = lambda x: A.quad_noise(x, m)
    mgf = lambda s: A.mgf_cumulants(s, phi_in, D, S, SQ2, 7.0)
    k = mgf(0.0)
    sig = math.sqrt(k[2])
    dN = sig / 20
    sp = A.SaddlepointDensity.from_mgf(np.arange(1000.0, 8001.0, 200.0), mgf)
    delay = A.em_classical_shift(phi_in, dN)
    nb, lo, hi = 64, k[1] + 2 * sig, k[1] + 18 * sig
    edges = lo + (hi - lo) / nb * np.arange(nb + 1)
    P = np.array([sp.bin_average(edges[j] - delay, edges[j + 1] - delay)
                  if sp.K1(sp.s[0]) < edges[j] - delay and edges[j + 1] - delay < sp.K1(sp.s[-1]) else np.nan
                  for j in range(nb)])
    sig_cl = PB.classical_sigma(m, phi_in)
    target = PB.classical_duration(0.0, 1.0, phi_in) + 8 * sig_cl
    n = 40000
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    res = {}
    for p in (1.0, 3.0):
        amp = PB.tune_amplitude(p, target, phi_in)
        prm = nat.make_params(precision="f64", m=m, n_max=hi, bias_p=p)
        nat.fpt_simulate(prm, n, phi_in, SQ2, math.inf, dN, amp, 0, N, lw)
        r = nat.fpt_pearson(N, lw)
        bins = nat.empty_bins(nb * N_SUB)
        counts = nat.empty_counts(1)
        nat.fpt_histogram(N, lw, nb, lo, hi, bins, counts, n_sub=N_SUB)
        est = nat.empty_estimates(nb)
        nat.fpt_estimate(bins, nb, lo, hi, n, est, n_sub=N_SUB)
        torch.cuda.synchronize()
        res[p] = (nat.estimates_to_dict(est), abs(r["r"]))
    e1, r1 = res[1.0]
    e3, r3 = res[3.0]
    use = (e3["count"] >= 400) & (e1["count"] >= 400) & np.isfinite(P)
    d3 = np.log(e3["p_direct"][use] / P[use])
    s3 = e3["se_direct"][use] / e3["p_direct"][use]
    d1 = np.log(e1["p_lognormal"][use] / P[use])
    s1 = np.hypot(0.5 * (e1["eps_lo"][use] + e1["eps_hi"][use]) / e1["p_lognormal"][use],
                  1 / np.sqrt(e1["count"][use]))
    z = (0.5 * (edges[1:] + edges[:-1]) - k[1]) / sig
    print(f"|r| p = 1: {r1:.4f}, p = 3: {r3:.6f}; {use.sum()} common bins, z {z[use].min():.1f}..{z[use].max():.1f}, "
          f"P down to {P[use].min():.1e}")
    print(f"p = 3 naive: max |dev|/se {np.max(np.abs(d3) / s3):.2f}, median relative error {np.median(s3):.4f}; "
          f"p = 1 lognormal: mean dev {np.mean(d1):+.4f}, max |dev|/err {np.max(np.abs(d1) / s1):.2f}, "
          f"median relative error {np.median(s1):.4f}")
    assert r3 > 0.9999 > r1
    assert use.sum() >= 8
    assert np.all(np.abs(d3) <= 4 * s3 + 0.01), np.max(np.abs(d3) / (4 * s3 + 0.01))
    assert np.median(s3) < np.median(s1)
