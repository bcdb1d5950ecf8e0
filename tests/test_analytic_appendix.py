"""Pins from the paper's appendices, checked against independent numerics and
the FP64 oracle (CPU only).

Appendix A (quadratic inflation, reflecting wall): the poles Lambda_n from the
pole equation A = B (Eq. (A.16), confluent hypergeometric functions) equal the
decay rates of the finite-difference generator; P(N) and Q(N) summed over the
poles with the residues of Eq. (A.18) equal the survival PDE's, and the
oracle's weighted tail agrees with them.

Appendix A without a wall (phi_uv -> infinity): the characteristic function
g(t, phi)/g(t, phi_end) has the mean of Eq. (19) and chi(0) = 1; the density
from the branch-cut integral (Eq. (A.28), prefactor 1/pi) is positive, its
survival function equals the survival PDE's with a far wall where the wall no
longer matters, its own derivative matches the density, the quadrature has
converged, and the far tail approaches the N^{-3/2} e^{-v0 N/4} law the
appendix derives, with a 1/N correction.

Appendix B: the Edgeworth expansion of Eq. (B.10) with He_3 = x^3 - 3x has the
moments it is built from (the printed He_3 = x^2 - 1 would change the
variance); the cumulants from the backward equations match the oracle's runs,
and near the peak the Edgeworth density fits the oracle's histogram where the
Gaussian does not.
"""
import math
import threading

import numpy as np
import pytest

import analytic as A
import oracle

pytest.importorskip("mpmath")
SQ2 = math.sqrt(2.0)
UV = 12.0  # reflecting wall for the drift-dominated cumulants (never reached)


def _fns(m, b=0.0):
    return (lambda x: A.quad_drift(x, b, m)), (lambda x: A.quad_noise(x, m))


@pytest.mark.parametrize("phi_uv,ref", [(9.0, (0.25138, 0.48839)), (math.sqrt(42.0), (0.6528, 1.0978))])
def test_pole_equation_matches_generator_eigenvalues(phi_uv, ref):
    poles = A.quad_poles(1.0, phi_uv, 3)
    lam = np.array([p[0] for p in poles])
    D, S = _fns(1.0)
    eig = A.generator_eigenvalues(D, S, SQ2, phi_uv, k=3, n=20001)
    np.testing.assert_allclose(lam, eig, rtol=2e-6)
    np.testing.assert_allclose(lam[:2], ref, rtol=2e-4)
    # Lambda_0 = v0/4 (Eq. (A.24)) does not hold with a wall this close: v0/4 = 5.3e-4
    assert lam[0] > 100 * (1.0 / (48 * math.pi ** 2)) / 4


def test_pole_expansion_matches_survival_pde():
    Ns = [30.0, 40.0, 60.0]
    P, Q, lam, a = A.quad_tail_from_poles(1.0, 9.0, 8.0, Ns, n_poles=12)
    assert np.all(np.diff(lam) > 0) and np.all(lam > 0)
    D, S = _fns(1.0)
    Qp = A.survival_pde(8.0, D, S, SQ2, 9.0, Ns, n=8001, dN=1e-3)
    np.testing.assert_allclose(Q, Qp, rtol=4e-3)
    # the far tail is the leading exponential (at N = 30 the next pole still adds 0.5 %)
    np.testing.assert_allclose(P[1:], lam[0] * Q[1:], rtol=1e-3)
    assert abs(P[0] / (lam[0] * Q[0]) - 1) < 2e-2
    assert math.isclose(Q[1], 1.0952e-3, rel_tol=1e-3)


def test_oracle_weighted_tail_matches_pole_expansion():
    """Biased oracle runs (b = 0.4, dN = 5e-4) reproduce Q(40) = P(N > 40) of the
    pole expansion within their statistical error and the O(sqrt(dN)) step bias."""
    P, Q, _, _ = A.quad_tail_from_poles(1.0, 9.0, 8.0, [40.0], n_poles=12)
    n, threads = 3200, 16
    res = [None] * threads

    def work(t):
        r = oracle.make_run(m=1.0, phi_in=8.0, phi_uv=9.0, dN=5e-4, b=0.4, n_max=60.0, seed=5,
                            traj_offset=t * (n // threads))
        res[t] = oracle.simulate(r, n // threads)
    ts = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    N = np.concatenate([r[0] for r in res])
    lw = np.concatenate([r[1] for r in res])
    x = np.where(N > 40.0, np.exp(lw), 0.0)
    est, se = x.mean(), x.std() / math.sqrt(n)
    assert abs(est - Q[0]) < 4 * se + 0.02 * Q[0], (est, se, Q[0])


def test_edgeworth_moments_fix_he3():
    mu, sig, g, k = 8.5, 0.6, 0.37, 0.65
    x = np.linspace(mu - 12 * sig, mu + 12 * sig, 200001)
    p = A.edgeworth_pdf(x, mu, sig, g, k)
    z = (x - mu) / sig
    mom = lambda f: np.trapezoid(f * p, x)
    assert math.isclose(mom(1.0), 1.0, rel_tol=1e-9)
    assert math.isclose(mom(x), mu, rel_tol=1e-9)
    assert math.isclose(mom(z ** 2), 1.0, rel_tol=1e-8)
    assert math.isclose(mom(z ** 3), g, rel_tol=1e-7)
    assert math.isclose(mom(z ** 4), 3 + k, rel_tol=1e-7)
    # with the printed He_3 = x^2 - 1 the variance would be 1 + g/3
    gauss = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi * sig * sig)
    wrong = gauss * (1 + g / 6 * (z ** 2 - 1) + k / 24 * A.hermite_he(4, z) + g ** 2 / 72 * A.hermite_he(6, z))
    assert abs(np.trapezoid(z ** 2 * wrong, x) - 1.0) > 0.1


@pytest.fixture(scope="module")
def interim_runs():
    """m = 0.3, phi_in = 6 (no wall): sigma_N = 0.61, skewness 0.37 — oracle
    runs with dN = 2e-3 over 16 threads."""
    n, threads = 16000, 16
    res = [None] * threads

    def work(t):
        r = oracle.make_run(m=0.3, phi_in=6.0, dN=2e-3, b=0.0, n_max=40.0, seed=9,
                            traj_offset=t * (n // threads))
        res[t] = oracle.simulate(r, n // threads)
    ts = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return np.concatenate([r[0] for r in res])


def test_backward_cumulants_match_oracle(interim_runs):
    N = interim_runs
    assert np.all(np.isfinite(N))
    D, S = _fns(0.3)
    # a wall at 12, which runs from 6 do not reach in drift domination, keeps the
    # far field of the finite differences away from the cumulants (converged to
    # 6 digits in grid size and wall position up to 20)
    k1, k2, k3, k4 = A.backward_cumulants(6.0, D, S, SQ2, UV, n=20001)
    mean_fd, var_fd = A.backward_moments_fd(6.0, D, S, SQ2, UV, n=20001)
    assert math.isclose(k1, mean_fd, rel_tol=1e-7) and math.isclose(k2, var_fd, rel_tol=1e-4)
    n = N.size
    c = N - N.mean()
    m2, m3, m4 = np.mean(c ** 2), np.mean(c ** 3), np.mean(c ** 4)
    g_s, k_s = m3 / m2 ** 1.5, m4 / m2 ** 2 - 3
    g, k = k3 / k2 ** 1.5, k4 / k2 ** 2
    assert abs(N.mean() - k1) < 4 * math.sqrt(k2 / n) + 2e-3
    assert abs(m2 / k2 - 1) < 4 * math.sqrt(2.0 / n) * math.sqrt(1 + k / 2)
    assert abs(g_s - g) < 4 * math.sqrt(6.0 / n), (g_s, g)
    assert abs(k_s - k) < 4 * math.sqrt(24.0 / n), (k_s, k)
    assert g > 0.3  # the skewness is resolved: ~20 standard errors


def test_edgeworth_fits_the_peak(interim_runs):
    """Within 2.5 sigma of the mean the Edgeworth density (cumulants from the
    backward equations) is consistent with the oracle's histogram (chi^2 per
    bin ~ 1) while the Gaussian with the same mean and variance is not."""
    N = interim_runs
    D, S = _fns(0.3)
    k1, k2, k3, k4 = A.backward_cumulants(6.0, D, S, SQ2, UV, n=20001)
    sig = math.sqrt(k2)
    edges = np.linspace(k1 - 2.5 * sig, k1 + 2.5 * sig, 41)
    cnt, _ = np.histogram(N, bins=edges)
    w = edges[1] - edges[0]
    mid = 0.5 * (edges[1:] + edges[:-1])
    exp_e = N.size * w * A.edgeworth_pdf(mid, k1, sig, k3 / sig ** 3, k4 / k2 ** 2)
    exp_g = N.size * w * A.edgeworth_pdf(mid, k1, sig, 0.0, 0.0)
    chi_e = np.sum((cnt - exp_e) ** 2 / exp_e) / cnt.size
    chi_g = np.sum((cnt - exp_g) ** 2 / exp_g) / cnt.size
    assert chi_e < 2.0, chi_e
    assert chi_g > 2 * chi_e and chi_g > 3.0, (chi_g, chi_e)


def test_no_wall_branch_cut_integral():
    import mpmath as mp
    m, phi = 1.0, math.sqrt(42.0)
    v0 = m * m / (48 * math.pi ** 2)
    y0 = v0 / 4
    # the closed-form characteristic function: chi(0) = 1 and the mean of Eq. (19)
    h = 1e-6
    lnM = lambda s: float(mp.log(mp.re(A.no_wall_chi(-1j * s, m, phi))))
    assert abs(lnM(0.0)) < 1e-30
    mean = (lnM(h) - lnM(-h)) / (2 * h)
    assert abs(mean / A.mean_fpt_quad(phi, m) - 1) < 1e-8, mean
    P, Q = A.no_wall_branch_cut(m, phi, 6.0, nodes=600)
    N = np.array([6.0, 8.0, 10.0, 15.0, 20.0, 30.0])
    # survival PDE with the wall at 20 (a wall at 30 changes these by < 1e-5)
    D, S = _fns(m)
    Qp = A.survival_pde(phi, D, S, SQ2, 20.0, np.concatenate([[0.0], N]), n=6001, dN=2e-3)[1:]
    np.testing.assert_allclose(Q(N), Qp, rtol=3e-3)
    # the pair is consistent: P = -dQ/dN
    dq = (Q(N - 1e-4) - Q(N + 1e-4)) / 2e-4
    np.testing.assert_allclose(dq, P(N), rtol=1e-6)
    # converged in the number of nodes
    P2, _ = A.no_wall_branch_cut(m, phi, 6.0, nodes=900)
    far = np.array([6.0, 10.0, 30.0, 73.0, 300.0, 3000.0])
    np.testing.assert_allclose(P(far), P2(far), rtol=1e-9)
    # positive, and the far tail N^{-3/2} e^{-v0 N / 4} A1 / sqrt(pi v0), A1 = lim Im chi / kappa
    grid = np.geomspace(6.0, 3e4, 60)
    assert np.all(P(grid) > 0)
    s = 1e-4
    A1 = A.no_wall_im_chi_on_cut(y0 + s * s, m, phi) / math.sqrt(4 * s * s / v0)
    r = lambda n: P(n)[0] * n ** 1.5 * math.exp(y0 * n) / (A1 / math.sqrt(math.pi * v0))
    r1, r3 = r(1e4) - 1, r(3e4) - 1
    assert 0 < r3 < 0.05 and 2.5 < r1 / r3 < 3.5, (r1, r3)
