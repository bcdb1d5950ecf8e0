"""The analytic helpers pinned against each other and against exact facts:
two independent solutions of the mean first-passage time, the survival
function integrating to the mean, and the inverse-Gaussian moments."""
import math

import numpy as np

import analytic as A

SQ2 = math.sqrt(2.0)


def test_quadrature_and_finite_differences_agree():
    for phi_in, m, b, uv in ((3.0, 1.0, 0.0, 300.0), (8.0, 1.0, 0.0, 9.0), (8.0, 1.0, 0.4, 9.0),
                             (3.0, 1.0, 1.0, 4.0)):
        q = A.mean_fpt_quad(phi_in, m, b=b, phi_uv=(math.inf if uv == 300.0 else uv))
        fd, _ = A.backward_moments_fd(phi_in, lambda x: A.quad_drift(x, b, m),
                                      lambda x: A.quad_noise(x, m), SQ2, uv, n=100001)
        assert abs(q - fd) < 2e-5 * q, (phi_in, m, b, uv, q, fd)


def test_classical_limit_of_mean():
    """Drift domination: <N> -> N_cl = (phi_in^2 - phi_end^2)/4 (§3, phi_in = sqrt 42 gives 10)."""
    assert abs(A.mean_fpt_quad(math.sqrt(42.0), 0.001) - 10.0) < 1e-5
    assert abs(A.mean_fpt_quad(6.0, 0.01) - 8.5) < 1e-4


def test_survival_function_integrates_to_mean():
    """E[N] = int_0^inf P(N > t) dt."""
    D = lambda x: A.quad_drift(x, 0.0, 1.0)
    S = lambda x: A.quad_noise(x, 1.0)
    grid = np.arange(0.0, 200.0, 0.05)
    Q = A.survival_pde(8.0, D, S, SQ2, 9.0, grid, n=2001, dN=5e-3)
    assert np.all(np.diff(Q) <= 1e-12) and Q[0] == 1.0
    integral = np.trapezoid(Q, grid)
    mean = A.mean_fpt_quad(8.0, 1.0, phi_uv=9.0)
    assert abs(integral - mean) < 2e-3 * mean


def test_survival_tail_reference_value():
    """P(N > 40) for m = 1, phi_in = 8, phi_uv = 9 (the far-tail event of the
    diffusion-dominated workload), converged in the grid."""
    D = lambda x: A.quad_drift(x, 0.0, 1.0)
    S = lambda x: A.quad_noise(x, 1.0)
    q1 = A.survival_pde(8.0, D, S, SQ2, 9.0, [40.0], n=2001, dN=4e-3)[0]
    q2 = A.survival_pde(8.0, D, S, SQ2, 9.0, [40.0], n=4001, dN=2e-3)[0]
    assert abs(q1 - q2) < 0.01 * q2
    assert 1.0e-3 < q2 < 1.2e-3


def test_inverse_gaussian_moments():
    ig = A.inverse_gaussian(2.0, 0.5, 0.3)
    assert abs(ig.mean() - 4.0) < 1e-12
    assert abs(ig.var() - 2.0 * 0.3**2 / 0.5**3) < 1e-12
