"""Host helpers of the power-law bias search (§3.4): the classical duration
against its closed form at A = 0 and against scipy quadrature, the amplitude
tuning, and the small-noise sigma_N against the backward-equation variance."""
import math

import numpy as np
import pytest

import analytic as A
from paper_2206_11234_gb300 import power_bias as PB

SQ2 = math.sqrt(2.0)


def test_classical_duration_closed_form_and_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    for p in (0.0, 1.0, 3.0, 4.5):
        assert math.isclose(PB.classical_duration(0.0, p, 6.0), (36.0 - 2.0) / 4.0, rel_tol=1e-13)
    for p, amp in ((3.0, 1e-4), (1.0, 0.01), (0.0, 0.1), (4.5, 2e-6)):
        ref = integrate.quad(lambda x: 1.0 / (2.0 / x - amp * x ** p), SQ2, 6.0, epsabs=0, epsrel=1e-13)[0]
        assert math.isclose(PB.classical_duration(amp, p, 6.0), ref, rel_tol=1e-10)
    assert PB.classical_duration(PB.max_amplitude(3.0, 6.0), 3.0, 6.0) == math.inf


@pytest.mark.parametrize("p", [0.0, 1.0, 2.0, 3.0, 4.0, 5.0])
def test_tune_amplitude_hits_the_target(p):
    target = 8.5 + 8 * PB.classical_sigma(0.001, 6.0)
    amp = PB.tune_amplitude(p, target, 6.0)
    assert 0 < amp < PB.max_amplitude(p, 6.0)
    assert math.isclose(PB.classical_duration(amp, p, 6.0), target, rel_tol=1e-9)


def test_classical_sigma_matches_backward_equation():
    """m = 0.01, phi_in = 6: Var N from the second backward equation (finite
    differences) and the small-noise integral agree to O(m^2) corrections."""
    m = 0.01
    D = lambda x: A.quad_drift(x, 0.0, m)
    S = lambda x: A.quad_noise(x, m)
    _, var = A.backward_moments_fd(6.0, D, S, SQ2, 8.0, n=40001)
    assert math.isclose(PB.classical_sigma(m, 6.0), math.sqrt(var), rel_tol=5e-3)
    assert math.isclose(PB.classical_sigma(m, 6.0), 0.02026, rel_tol=2e-3)
