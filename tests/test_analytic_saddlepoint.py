"""Pins of the far-tail reference for drift domination (CPU only): the
cumulant generating function K(s) = ln E[e^{sN}] from the Riccati form of the
backward equation (Appendix A, Eq. (A.2), on the real axis), its saddle-point
density, and the Euler-Maruyama delay of the classical duration.

* At s = 0 the derivatives of K are the cumulants of the backward recursion
  (an independent finite-difference solve).
* Brownian motion with drift (the constant test model): K(s) in closed form,
  and the saddle-point density is the inverse-Gaussian density, exact for
  this law (Daniels 1980), far into the tail.
* Quadratic inflation with a wall: K(s) equals the logarithm of Appendix A's
  hypergeometric solution, below and above s = v0/4 (real and imaginary alpha).
* The delay of the noise-free map, dN/2 ln(phi_in/phi_end) to first order, is
  the shift of the oracle's mean first-passage time in drift domination.
"""
import math
import threading

import numpy as np
import pytest

import analytic as A
import oracle

SQ2 = math.sqrt(2.0)


def _quad(m):
    return (lambda x: A.quad_drift(x, 0.0, m)), (lambda x: A.quad_noise(x, m))


def test_derivatives_at_zero_are_the_backward_cumulants():
    for m, phi_in, top in ((0.01, 6.0, 7.0), (0.3, 6.0, 12.0)):
        D, S = _quad(m)
        K = A.mgf_cumulants(0.0, phi_in, D, S, SQ2, top)
        ref = A.backward_cumulants(phi_in, D, S, SQ2, top, n=20001)
        assert K[0] == 0.0
        np.testing.assert_allclose(K[1:], ref, rtol=2e-6)


def test_derivatives_are_consistent_with_differences_of_k():
    D, S = _quad(0.01)
    h = 0.5
    for s in (-150.0, 300.0, 700.0):
        k = [A.mgf_cumulants(s + j * h, 6.0, D, S, SQ2, 7.0) for j in (-2, -1, 0, 1, 2)]
        c = k[2]
        d1 = (k[0][0] - 8 * k[1][0] + 8 * k[3][0] - k[4][0]) / (12 * h)
        d2 = (k[0][1] - 8 * k[1][1] + 8 * k[3][1] - k[4][1]) / (12 * h)
        d3 = (k[0][2] - 8 * k[1][2] + 8 * k[3][2] - k[4][2]) / (12 * h)
        assert math.isclose(d1, c[1], rel_tol=1e-9)
        assert math.isclose(d2, c[2], rel_tol=1e-7)
        assert math.isclose(d3, c[3], rel_tol=1e-5)


def test_constant_model_closed_form():
    a0, s0, dist = -1.0, 0.3, 1.0
    D, S = (lambda x: a0 + 0.0 * x), (lambda x: s0 + 0.0 * x)
    # wall 6 above the start: not felt even by the tilted process at s = 5,
    # whose drift toward the barrier is only sqrt(a0^2 - 2 s0^2 s) = 0.32
    # (escape ~ exp(-2 * 0.32 * 6 / s0^2) = e^-42)
    for s in (-20.0, -3.0, 0.0, 1.0, 3.0, 5.0):
        K = A.mgf_cumulants(s, 1.0 + dist, D, S, 1.0, 1.0 + dist + 6.0)
        ref = A.constant_model_log_mgf(s, dist, -a0, s0)
        assert math.isclose(K[0], ref, rel_tol=1e-9, abs_tol=1e-12), (s, K[0], ref)
        # K'(s) = (d / sqrt(a0^2 - 2 s0^2 s)) from the closed form
        assert math.isclose(K[1], dist / math.sqrt(a0 * a0 - 2 * s0 * s0 * s), rel_tol=1e-8)


def test_saddlepoint_is_exact_for_the_inverse_gaussian():
    """The saddle-point density of an inverse-Gaussian law is exact (its first
    correction, lambda_4/8 - 5 lambda_3^2/24, vanishes for this law), so both
    forms equal the exact density from 2 sigma below the mean to 11 sigma above
    it, to 1e-9 with the generating function evaluated at each saddle point
    (N = mean + 11 sigma needs s = 39, near the end of K(s) at
    a0^2/(2 s0^2) = 50)."""
    a0, s0, dist = -1.0, 0.1, 1.0
    D, S = (lambda x: a0 + 0.0 * x), (lambda x: s0 + 0.0 * x)
    grid = np.arange(-60.0, 41.0, 5.0)
    sp = A.SaddlepointDensity.from_mgf(grid, lambda s: A.mgf_cumulants(s, 2.0, D, S, 1.0, 3.0))
    law = A.inverse_gaussian(dist, -a0, s0)
    mean, sd = law.mean(), law.std()
    N = np.linspace(mean - 2 * sd, mean + 11 * sd, 8)
    exact = law.pdf(N)
    assert exact[-1] < 1e-10
    np.testing.assert_allclose(sp.pdf(N, exact=True), exact, rtol=1e-9)
    np.testing.assert_allclose(sp.pdf(N, correction=False, exact=True), exact, rtol=1e-9)


@pytest.mark.parametrize("s", [-0.6, -0.05, 0.0003, 0.12, 0.24])
def test_quadratic_with_wall_matches_appendix_a(s):
    """m = 1, phi_in = 8, wall at 9: v0/4 = 5.3e-4 and the leading pole 0.2514
    bracket the positive s."""
    pytest.importorskip("mpmath")
    D, S = _quad(1.0)
    K = A.mgf_cumulants(s, 8.0, D, S, SQ2, 9.0)
    ref = A.quad_log_mgf_appendix_a(s, 1.0, 8.0, SQ2, 9.0)
    assert math.isclose(K[0], ref, rel_tol=1e-8, abs_tol=1e-10), (K[0], ref)


def test_saddlepoint_density_of_drift_domination():
    """m = 0.01, phi_in = 6: normalised, near the peak equal to the Edgeworth
    density of Appendix B built from the same cumulants, and the table's
    interpolation exact to 1e-5 far into the tail."""
    D, S = _quad(0.01)
    grid = np.arange(-300.0, 751.0, 50.0)
    sp = A.SaddlepointDensity.from_mgf(grid, lambda s: A.mgf_cumulants(s, 6.0, D, S, SQ2, 7.0))
    k1, k2, k3, k4 = A.mgf_cumulants(0.0, 6.0, D, S, SQ2, 7.0)[1:]
    sig = math.sqrt(k2)
    x = np.linspace(k1 - 5 * sig, k1 + 5 * sig, 2001)
    assert abs(np.trapezoid(sp.pdf(x), x) - 1) < 1e-5
    z = np.linspace(k1 - 2 * sig, k1 + 2 * sig, 9)
    np.testing.assert_allclose(sp.pdf(z), A.edgeworth_pdf(z, k1, sig, k3 / sig ** 3, k4 / k2 ** 2), rtol=2e-4)
    # the interpolated table (step 50 in s: K to ~1e-6) against saddle points
    # solved exactly, out to 13 sigma
    far = k1 + sig * np.array([-4.0, 6.0, 13.0])
    np.testing.assert_allclose(sp.pdf(far), sp.pdf(far, exact=True), rtol=1e-5)


def test_em_delay_of_the_classical_duration():
    """The noise-free map lags N_cl by dN/2 ln(phi_in/phi_end) to first order,
    and the oracle's mean first-passage time (m = 0.01, phi_in = 6, dN = 1e-2,
    16000 runs) is K'(0) plus that delay: 7.2e-3, 45 standard errors."""
    for dN in (1e-2, 1e-3, 1e-4):
        assert math.isclose(A.em_classical_shift(6.0, dN), 0.5 * dN * math.log(6.0 / SQ2), rel_tol=4 * dN)
    n, threads, dN = 16000, 16, 1e-2
    res = [None] * threads

    def work(t):
        r = oracle.make_run(m=0.01, phi_in=6.0, dN=dN, b=0.0, n_max=12.0, seed=17, traj_offset=t * (n // threads))
        res[t] = oracle.simulate(r, n // threads)[0]
    ts = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    N = np.concatenate(res)
    D, S = _quad(0.01)
    k1 = A.mgf_cumulants(0.0, 6.0, D, S, SQ2, 7.0)[1]
    delay = A.em_classical_shift(6.0, dN)
    se = N.std() / math.sqrt(n)
    assert abs(N.mean() - k1 - delay) < 4 * se, (N.mean() - k1, delay, se)
    assert delay > 30 * se


def test_characteristic_function_of_brownian_motion_with_drift():
    """ln E[e^{iwN}] = (d/s0^2)(|a0| - sqrt(a0^2 - 2 i s0^2 w)) (principal root)."""
    a0, s0, dist = -1.0, 0.3, 1.0
    D, S = (lambda x: a0 + 0.0 * x), (lambda x: s0 + 0.0 * x)
    for w in (0.5, 3.0, 12.0):
        got = A.log_characteristic_function(w, 1.0 + dist, D, S, 1.0, 1.0 + dist + 6.0)
        ref = dist / s0 ** 2 * (-a0 - np.sqrt(complex(a0 * a0, -2 * s0 * s0 * w)))
        assert abs(got - ref) < 1e-8 * abs(ref), (w, got, ref)


def test_characteristic_function_matches_cumulants_and_saddle_point():
    """m = 0.01, phi_in = 6: at small w ln chi = sum_k kappa_k (i w)^k / k! to
    O(w^5); the Fourier density equals the saddle-point density from -3 to +5
    sigma (two inversions of the same backward equation)."""
    D, S = _quad(0.01)
    k = A.mgf_cumulants(0.0, 6.0, D, S, SQ2, 7.0)
    w = 2.0
    series = sum(k[j] * (1j * w) ** j / math.factorial(j) for j in range(1, 5))
    got = A.log_characteristic_function(w, 6.0, D, S, SQ2, 7.0)
    assert abs(got - series) < 1e-6, (got, series)
    sig = math.sqrt(k[2])
    # dw = 0.3 / sigma puts the aliases 21 sigma away; |chi| < 1e-11 beyond 7.5 / sigma
    fd = A.FourierDensity(0.3 / sig, 26, lambda x: A.log_characteristic_function(x, 6.0, D, S, SQ2, 7.0))
    sp = A.SaddlepointDensity.from_mgf(np.arange(-300.0, 326.0, 25.0),
                                       lambda s: A.mgf_cumulants(s, 6.0, D, S, SQ2, 7.0))
    N = k[1] + sig * np.array([-3.0, -1.0, 0.0, 1.5, 3.0, 5.0])
    np.testing.assert_allclose(fd.pdf(N), sp.pdf(N), rtol=2e-4)
