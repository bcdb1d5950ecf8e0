"""Pins of the oracle's biased Euler–Maruyama first-passage simulation against
what the paper and the mathematics fix (closed forms, backward equations,
exact identities, brute-force likelihood ratios).  CPU only."""
import math

import numpy as np
import pytest
import scipy.stats as stats

import analytic as A
import oracle
from paper_2206_11234_gb300 import workloads as W

SQ2 = math.sqrt(2.0)


def _quad_fns(m):
    return (lambda x: A.quad_drift(x, 0.0, m)), (lambda x: A.quad_noise(x, m))


def test_zero_bias_log_weight_is_exactly_zero():
    """With B = 0 every weight is 1 (§2.2, below Eq. (16))."""
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=0.0, n_max=6.0)
    N, lw, steps = oracle.simulate(r, 2000)
    assert np.all(lw == 0.0)
    assert np.all(np.isfinite(N)) and np.all(steps > 0)


def test_start_at_or_below_end_gives_zero_time():
    for phi_in in (SQ2, 1.0):
        r = oracle.make_run(m=1.0, phi_in=phi_in, dN=1e-3, b=1.0, n_max=6.0)
        N, lw, steps = oracle.simulate(r, 10)
        assert np.all(N == 0.0) and np.all(lw == 0.0) and np.all(steps == 0)


def test_invalid_arguments_rejected():
    bad = [dict(dN=0.0), dict(dN=-1e-3), dict(n_max=math.inf), dict(phi_uv=2.0),
           dict(dN=math.nan)]
    for kw in bad:
        args = dict(m=1.0, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0)
        args.update(kw)
        with pytest.raises(ValueError):
            oracle.simulate(oracle.make_run(**args), 4)


def test_constant_model_matches_inverse_gaussian():
    """Constant drift a0 < 0 and noise s0: the first-passage time over a distance
    d is inverse-Gaussian; discrete monitoring (the first step index M at or
    past the barrier) shifts the barrier by 0.5826 s0 sqrt(dN)
    (Broadie–Glasserman–Kou).  The interpolated time N lies within one step
    before M dN."""
    a0, s0, d = -1.0, 0.5, 1.0
    for dN, n in ((1e-2, 20000), (1e-3, 20000)):
        r = oracle.make_run(model=oracle.MODEL_CONSTANT, a0=a0, s0=s0, phi_in=1.0 + d,
                            phi_end=1.0, dN=dN, b=0.0, n_max=30.0)
        N, lw, steps = oracle.simulate(r, n)
        assert np.all(np.isfinite(N))
        T = steps * dN
        assert np.all(N <= T) and np.all(N > T - dN)
        ig = A.inverse_gaussian(A.bgk_distance(d, s0, dN), -a0, s0)
        se = math.sqrt(ig.var() / n)
        assert abs(T.mean() - ig.mean()) < 4 * se
        assert stats.kstest(T, ig.cdf).pvalue > 1e-3
        if dN == 1e-2:
            # without the continuity correction the law is detectably wrong
            ig0 = A.inverse_gaussian(d, -a0, s0)
            assert abs(T.mean() - ig0.mean()) > 4 * se


def test_constant_model_biased_law_and_weights():
    """Biased sampling: the unweighted times follow the law with drift a0 + b s0;
    the weighted ones reproduce the target law (Eq. (16)); and the log-weight is
    fixed by the end point: ln w = -b (phi_M - phi_in)/s0 + (b (a0 + b s0)/s0 - b^2/2) M dN."""
    a0, s0, d, b, dN, n = -1.0, 0.5, 1.0, 0.8, 1e-3, 20000
    r = oracle.make_run(model=oracle.MODEL_CONSTANT, a0=a0, s0=s0, phi_in=1.0 + d, phi_end=1.0,
                        dN=dN, b=b, n_max=40.0)
    N, lw, steps = oracle.simulate(r, n)
    assert np.all(np.isfinite(N))
    de = A.bgk_distance(d, s0, dN)
    sample = A.inverse_gaussian(de, -(a0 + b * s0), s0)
    assert stats.kstest(steps * dN, sample.cdf).pvalue > 1e-3
    target = A.inverse_gaussian(de, -a0, s0)
    w = np.exp(lw)
    for t in (0.5, 0.8, 1.0, 1.5, 2.5):
        x = w * (N <= t)
        assert abs(x.mean() - target.cdf(t)) < 4 * x.std() / math.sqrt(n) + 2e-3
    for i in range(5):
        phi, xi, bu, Ni, lwi = oracle.path(r, i, 100000)
        M = xi.size
        closed = -b * (phi[-1] - phi[0]) / s0 + (b * (a0 + b * s0) / s0 - 0.5 * b * b) * M * dN
        assert abs(lwi - closed) < 1e-9 * (1 + abs(closed))


def test_log_weight_closed_form_for_constant_bias():
    """For constant b the per-step sum collapses: ln w = -b sqrt(dN) sum xi - b^2 M dN / 2."""
    b, dN = 1.0, 1e-3
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=dN, b=b, n_max=6.0)
    N, lw, steps = oracle.simulate(r, 8)
    for i in range(8):
        M = int(steps[i])
        xi = np.concatenate([oracle.normals4(0, i, 0, k) for k in range((M + 3) // 4)])[:M]
        inc = b * math.sqrt(dN) * np.abs(xi) + 0.5 * b * b * dN
        closed = -b * math.sqrt(dN) * math.fsum(xi) - 0.5 * b * b * M * dN
        assert abs(lw[i] - closed) <= 1e-12 * max(1.0, inc.sum())


@pytest.mark.parametrize("b", [0.7, 1.3])
def test_path_likelihood_ratio_fixes_the_weight_sign(b):
    """ln w equals ln p_T(X) - ln p_S(X) computed from the Gaussian step densities
    of Eqs. (13)-(14) by brute force; the overall sign printed in Eq. (15) would
    give the negative of this."""
    dN = 1e-3
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=dN, b=b, n_max=6.0)
    D, S = _quad_fns(1.0)
    for i in range(4):
        phi, xi, bu, Ni, lwi = oracle.path(r, i, 200000)
        ref = A.path_log_likelihood_ratio(phi, bu, D, S, dN)
        assert abs(lwi - ref) < 1e-8 * (1 + abs(ref)) + 1e-9 * xi.size
        assert abs(lwi + ref) > 1e-3  # the printed sign is distinguishable


def test_unbiased_mean_and_variance_match_backward_equations():
    """<N> from the double integral of §2.3 Eq. (19) and Var N from the second
    backward equation, for the quadratic model with no wall (m = 1, phi_in = 3)."""
    n, dN = 16384, 1e-3
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=dN, b=0.0, n_max=40.0)
    N, lw, _ = oracle.simulate(r, n)
    mean_q = A.mean_fpt_quad(3.0, 1.0)
    D, S = _quad_fns(1.0)
    mean_fd, var_fd = A.backward_moments_fd(3.0, D, S, SQ2, 300.0, n=100001)
    assert abs(mean_q - mean_fd) < 1e-5
    se = math.sqrt(var_fd / n)
    assert abs(N.mean() - mean_q) < 4 * se + 1e-3
    assert abs(N.var() - var_fd) < 5 * var_fd * math.sqrt(2.0 / n) * 2


def test_biased_means_with_wall_match_quadrature():
    """With a reflecting wall the sample process mean (unweighted) is Eq. (19)
    with D + B, and the self-normalised weighted mean is the b = 0 value."""
    n, dN, b = 8000, 1e-3, 1.0
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=dN, b=b, n_max=200.0)
    N, lw, _ = oracle.simulate(r, n)
    assert np.all(np.isfinite(N))
    ms = A.mean_fpt_quad(3.0, 1.0, b=b, phi_uv=4.0)
    D, S = (lambda x: A.quad_drift(x, b, 1.0)), (lambda x: A.quad_noise(x, 1.0))
    _, var_s = A.backward_moments_fd(3.0, D, S, SQ2, 4.0)
    assert abs(N.mean() - ms) < 4 * math.sqrt(var_s / n) + 2e-3
    w = np.exp(lw)
    mt = A.mean_fpt_quad(3.0, 1.0, b=0.0, phi_uv=4.0)
    est = np.sum(w * N) / np.sum(w)
    # delta-method standard error of the ratio estimator
    se = math.sqrt(np.mean((w * (N - est)) ** 2) / n) / np.mean(w)
    assert abs(est - mt) < 4 * se + 2e-3


def test_drift_dominated_mean():
    """m = 0.01, phi_in = 6: <N> = 8.50002 from Eq. (19); sigma_N ~ 0.02."""
    n, dN = 1500, 1e-3
    r = oracle.make_run(m=0.01, phi_in=6.0, dN=dN, b=0.0, n_max=10.0)
    N, _, _ = oracle.simulate(r, n)
    mq = A.mean_fpt_quad(6.0, 0.01)
    assert abs(mq - 8.50002) < 1e-4
    assert abs(N.mean() - mq) < 4 * N.std() / math.sqrt(n) + 1e-4


def test_mean_weight_is_one_even_with_censoring():
    """E_S[w] = 1 (w = p_T/p_S of the stopped path); censoring at a fixed step
    cap keeps this exact."""
    for n_max, n in ((6.0, 16384), (1.5, 16384)):
        r = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=1.0, n_max=n_max)
        N, lw, _ = oracle.simulate(r, n)
        w = np.exp(lw)
        assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(n)
        if n_max == 1.5:
            assert np.mean(~np.isfinite(N)) > 0.3


def test_reflection_keeps_paths_below_wall_and_weight_uses_drawn_noise():
    dN, b = 1e-3, 5.0  # b S > |D| near phi_in: the sample drift pushes into the wall
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=3.05, dN=dN, b=b, n_max=5.0)
    D, S = _quad_fns(1.0)
    n_reflect = 0
    for i in range(6):
        phi, xi, bu, Ni, lwi = oracle.path(r, i, 400000)
        assert phi.max() <= 3.05
        # the weight depends only on the drawn normals (constant b)
        closed = -b * math.sqrt(dN) * math.fsum(xi) - 0.5 * b * b * xi.size * dN
        assert abs(lwi - closed) < 1e-12 * (1 + np.abs(xi).sum())
        S_ = A.quad_noise(phi[:-1], 1.0)
        raw = phi[:-1] + (D(phi[:-1]) + b * S_) * dN + S_ * xi * math.sqrt(dN)
        n_reflect += int(np.sum(raw > 3.05))
    assert n_reflect > 0


def test_censoring_at_step_cap():
    dN = 1e-3
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=dN, b=0.0, n_max=0.01)
    N, lw, steps = oracle.simulate(r, 50)
    assert np.all(np.isinf(N)) and np.all(steps == oracle.step_cap(0.01, dN))


def test_trajectory_ids_shard_exactly():
    r = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0)
    N, lw, st = oracle.simulate(r, 64)
    r2 = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0, traj_offset=40)
    N2, lw2, st2 = oracle.simulate(r2, 24)
    assert np.array_equal(N[40:], N2) and np.array_equal(lw[40:], lw2)


def test_biased_and_direct_histograms_agree():
    """Importance sampling reproduces the direct estimate (§2.1 Eq. (9) vs
    §2.2 Eq. (16)) in bins both populate (>= 400 runs each)."""
    n, lo, hi, nb = 20000, 0.0, 6.0, 60
    width = (hi - lo) / nb
    r0 = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=0.0, n_max=6.0)
    r1 = oracle.make_run(m=1.0, phi_in=3.0, dN=1e-3, b=0.5, n_max=6.0, seed=1)
    N0, lw0, _ = oracle.simulate(r0, n)
    N1, lw1, _ = oracle.simulate(r1, n)
    b0, _ = oracle.histogram(N0, lw0, nb, lo, hi)
    b1, _ = oracle.histogram(N1, lw1, nb, lo, hi)
    compared = 0
    for j in range(nb):
        c0, c1 = b0[0, j, 7], b1[0, j, 7]
        if c0 < 400 or c1 < 400:
            continue
        p0 = c0 / (n * width)
        s0 = math.sqrt(c0) / (n * width)
        mx = b1[0, j, 0]
        p1 = math.exp(mx) * b1[0, j, 1] / (n * width)
        m2 = math.exp(2 * mx) * b1[0, j, 2] / n
        s1 = math.sqrt(max(m2 - (p1 * width) ** 2, 0.0) / n) / width
        assert abs(p0 - p1) < 4 * math.hypot(s0, s1), j
        compared += 1
    assert compared >= 8


# ---- power-law bias B = A_p phi^p (§3.4 Eq. (26)) ----

C0 = 1.0 / (2.0 * math.pi * math.sqrt(6.0))


def test_power_bias_p1_is_the_constant_bias():
    """p = 1 with A_1 = b c0 m is the bias B = b S of §2.3 Eq. (18)."""
    r1 = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=3.5, dN=1e-3, b=0.8, n_max=6.0)
    r2 = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=3.5, dN=1e-3, b=0.8 * C0, n_max=6.0, bias_p=1.0)
    a, b = oracle.simulate(r1, 300), oracle.simulate(r2, 300)
    assert np.array_equal(a[2], b[2])
    np.testing.assert_allclose(b[0], a[0], rtol=1e-13)
    np.testing.assert_allclose(b[1], a[1], rtol=0, atol=1e-12)


@pytest.mark.parametrize("p,amp", [(3.0, 0.004), (2.5, 0.01), (0.0, 0.3)])
def test_power_bias_weight_is_the_path_likelihood_ratio(p, amp):
    """ln w of a state-dependent bias equals ln p_T - ln p_S from the Gaussian
    step densities of Eqs. (13)-(14), step by step (brute force)."""
    dN = 1e-3
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=dN, b=amp, n_max=20.0, bias_p=p)
    D, S = _quad_fns(1.0)
    for i in range(3):
        phi, xi, bu, Ni, lwi = oracle.path(r, i, 400000)
        np.testing.assert_allclose(bu * S(phi[:-1]), amp * phi[:-1] ** p, rtol=1e-13)
        ref = A.path_log_likelihood_ratio(phi, bu, D, S, dN)
        assert abs(lwi - ref) < 1e-8 * (1 + abs(ref)) + 1e-9 * xi.size


def test_power_bias_means_and_unit_mean_weight():
    """Sample-process mean FPT from the backward equation with drift D + A phi^3
    (wall at 4), E[w] = 1, and the weighted mean equal to the b = 0 value."""
    n, dN, amp, p = 6000, 1e-3, 0.004, 3.0
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=dN, b=amp, n_max=200.0, bias_p=p)
    N, lw, _ = oracle.simulate(r, n)
    assert np.all(np.isfinite(N))
    Ds = lambda x: A.quad_drift(x, 0.0, 1.0) + amp * x ** p
    S = lambda x: A.quad_noise(x, 1.0)
    ms, vs = A.backward_moments_fd(3.0, Ds, S, SQ2, 4.0)
    assert abs(N.mean() - ms) < 4 * math.sqrt(vs / n) + 2e-3
    w = np.exp(lw)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(n)
    mt = A.mean_fpt_quad(3.0, 1.0, b=0.0, phi_uv=4.0)
    est = np.sum(w * N) / np.sum(w)
    se = math.sqrt(np.mean((w * (N - est)) ** 2) / n) / np.mean(w)
    assert abs(est - mt) < 4 * se + 2e-3


def test_power_bias_drift_dominated_classical_duration():
    """m = 0.01: the sample duration approaches the classical
    N_S,cl = int dphi / (2/phi - A_p phi^p) from phi_end to phi_in (§2.4)."""
    from scipy import integrate
    p, amp, dN = 3.0, 1e-4, 1e-3  # drift stays negative: amp < 2 / phi_in^(p+1)
    r = oracle.make_run(m=0.01, phi_in=6.0, dN=dN, b=amp, n_max=20.0, bias_p=p)
    N, lw, _ = oracle.simulate(r, 400)
    ncl = integrate.quad(lambda x: 1.0 / (2.0 / x - amp * x ** p), SQ2, 6.0, epsabs=1e-12, epsrel=1e-12)[0]
    assert ncl > 8.6  # the bias lengthens inflation by several sigma_N ~ 0.02
    assert abs(N.mean() / ncl - 1) < 5e-4


# ---- general potential V(phi) = sum_k c_k phi^k (§2.3 Eq. (17)) ----

def _poly_fns(c):
    """D = -V'/V and S = sqrt(V/3)/(2 pi) of the polynomial potential, numpy."""
    P = np.polynomial.Polynomial(c)
    dP = P.deriv()
    return (lambda x: -dP(x) / P(x)), (lambda x: np.sqrt(P(x) / 3.0) / (2 * math.pi))


def test_polynomial_model_reduces_to_quadratic():
    m = 0.7
    a = oracle.simulate(oracle.make_run(m=m, phi_in=3.0, phi_uv=3.5, dN=1e-3, b=0.7, n_max=6.0), 300)
    b = oracle.simulate(oracle.make_run(model=oracle.MODEL_POLYNOMIAL, poly=[0, 0, 0.5 * m * m], phi_in=3.0,
                                        phi_uv=3.5, dN=1e-3, b=0.7, n_max=6.0), 300)
    assert np.array_equal(a[2], b[2])
    np.testing.assert_allclose(b[0], a[0], rtol=1e-12)
    np.testing.assert_allclose(b[1], a[1], rtol=0, atol=1e-10)


@pytest.mark.parametrize("c,phi_in,phi_end,phi_uv,b", [
    ([0, 0, 0, 0, 0.25 * 0.05], 4.0, math.sqrt(8.0), 4.6, 0.0),         # quartic lambda phi^4 / 4
    ([0, 0, 0.5 * 0.3, 0, 0.25 * 0.02], 3.5, 1.6, 4.0, 0.5),            # phi^2 + phi^4 mix, biased
])
def test_polynomial_model_moments_and_weights(c, phi_in, phi_end, phi_uv, b):
    """<N> and Var N of the sample process from the backward equations with
    D + b S, and E[w] = 1 with the weighted mean equal to the unbiased one."""
    n, dN = 6000, 1e-3
    r = oracle.make_run(model=oracle.MODEL_POLYNOMIAL, poly=c, phi_in=phi_in, phi_end=phi_end, phi_uv=phi_uv, dN=dN,
                        b=b, n_max=200.0)
    N, lw, _ = oracle.simulate(r, n)
    assert np.all(np.isfinite(N))
    D, S = _poly_fns(c)
    ms, vs = A.backward_moments_fd(phi_in, lambda x: D(x) + b * S(x), S, phi_end, phi_uv)
    assert abs(N.mean() - ms) < 4 * math.sqrt(vs / n) + 3e-3 * ms
    assert abs(N.var() / vs - 1) < 4 * math.sqrt(2.0 / n) * 2
    w = np.exp(lw)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(n) + 1e-12
    mt, _ = A.backward_moments_fd(phi_in, D, S, phi_end, phi_uv)
    est = np.sum(w * N) / np.sum(w)
    se = math.sqrt(np.mean((w * (N - est)) ** 2) / n) / np.mean(w)
    assert abs(est - mt) < 4 * se + 3e-3 * mt
