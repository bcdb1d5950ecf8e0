"""Host side of the power-law bias search of arXiv:2206.11234 §3.4.

The bias B = A_p phi^p (Eq. (26)) is compared across p at equal displacement
of the sample distribution: A_p is chosen so that the classical duration of
the sample process lies a fixed number of standard deviations of the target
distribution past the target's classical duration, and each p is then scored
by |r|, Pearson's correlation of ln w with N (fpt_pearson): the more squeezed
the (N, w) cloud, the smaller the spread of the weights within a bin.

Quadratic inflation, M_Pl = 1: D = -2/phi, S = c0 m phi (§2.3 Eq. (17), §3
Eq. (25)), phi_end = sqrt(2).  These are parameter-selection helpers that run
on the host; the simulation itself is fpt_simulate with FPT_BIAS_POWER.
"""
import math

import numpy as np

PHI_END = math.sqrt(2.0)


def classical_duration(amp: float, p: float, phi_in: float, phi_end: float = PHI_END, nodes: int = 256) -> float:
    """N_S,cl = integral from phi_end to phi_in of dphi / (2/phi - A_p phi^p): the
    noise-free sample process (§2.4), Gauss-Legendre on `nodes` points.  Needs
    the sample drift to stay negative on the interval (amp < max_amplitude)."""
    if amp >= max_amplitude(p, phi_in, phi_end):
        return math.inf
    x, w = np.polynomial.legendre.leggauss(nodes)
    phi = 0.5 * (phi_in - phi_end) * x + 0.5 * (phi_in + phi_end)
    return float(0.5 * (phi_in - phi_end) * np.sum(w / (2.0 / phi - amp * phi ** p)))


def max_amplitude(p: float, phi_in: float, phi_end: float = PHI_END) -> float:
    """Largest A_p for which the sample drift -2/phi + A_p phi^p stays negative
    on [phi_end, phi_in] (beyond it runs can escape to large phi)."""
    return 2.0 / max(phi_in ** (p + 1.0), phi_end ** (p + 1.0))


def classical_sigma(m: float, phi_in: float, phi_end: float = PHI_END) -> float:
    """Standard deviation of N in the drift-dominated limit: the small-noise
    expansion of the second backward moment, Var N = integral of S^2 / |D|^3
    dphi = m^2 (phi_in^6 - phi_end^6) / (1152 pi^2) for the quadratic model."""
    return math.sqrt(m * m * (phi_in ** 6 - phi_end ** 6) / (1152.0 * math.pi ** 2))


def tune_amplitude(p: float, target: float, phi_in: float, phi_end: float = PHI_END, rtol: float = 1e-12) -> float:
    """A_p >= 0 with classical_duration(A_p, p) = target (bisection; the
    duration grows monotonically with A_p)."""
    lo, hi = 0.0, max_amplitude(p, phi_in, phi_end)
    if not classical_duration(0.0, p, phi_in, phi_end) <= target:
        raise ValueError("target below the unbiased classical duration")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if classical_duration(mid, p, phi_in, phi_end) < target:
            lo = mid
        else:
            hi = mid
        if hi - lo <= rtol * hi:
            break
    return 0.5 * (lo + hi)
