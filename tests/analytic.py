"""Closed forms and deterministic numerics that pin the oracle (test-only).

None of this is the method itself: these are the mathematical facts the
Monte Carlo must reproduce.

* ``mean_fpt_quad``: the mean first-passage time of the (biased) sample
  process as the double integral of §2.3 Eq. (19), with the inner exponent
  integrated in closed form for the quadratic model (§3 Eq. (25)).
* ``backward_moments_fd``: the same mean, and the second moment, from the
  backward (adjoint Fokker–Planck) equations (S^2/2) T'' + (D+B) T' = -f with
  T(phi_end) = 0 and T'(phi_uv) = 0 (absorbing end, reflecting wall; Appendix A
  boundary conditions), f = 1 for <N> and f = 2 <N> for <N^2> — a textbook
  result for exit times of diffusions, solved by second-order finite differences.
* ``survival_pde``: Q(phi, N) = P(first passage later than N), from
  dQ/dN = (S^2/2) Q'' + (D+B) Q' with the same boundary conditions and
  Q(phi, 0) = 1, by backward Euler (an M-matrix scheme, so 0 <= Q <= 1).
* ``inverse_gaussian``: first-passage law of Brownian motion with constant
  drift (the constant test model), via scipy.stats.invgauss, with the
  Broadie–Glasserman–Kou continuity correction for discrete monitoring.
"""
import math
import warnings

import numpy as np
import scipy.integrate as integrate
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.stats as stats

C0 = 1.0 / (2.0 * math.pi * math.sqrt(6.0))  # S = C0 * m * phi for V = m^2 phi^2 / 2
BGK_BETA = 0.5825971579390106  # -zeta(1/2) / sqrt(2 pi), Broadie–Glasserman–Kou (1997)


def quad_drift(phi, b, m):
    """D + B for the quadratic model with bias B = b * S."""
    return -2.0 / phi + b * C0 * m * phi


def quad_noise(phi, m):
    return C0 * m * phi


def mean_fpt_quad(phi_in, m, b=0.0, phi_end=math.sqrt(2.0), phi_uv=math.inf):
    """<N>_S(phi_in) from §2.3 Eq. (19) for the quadratic model.

    Inner exponent 2 int_{p1}^{p2} (D+B)/S^2 = (2/(C0 m)^2)(1/p2^2 - 1/p1^2)
    + (2 b/(C0 m)) ln(p2/p1).
    """
    a = 2.0 / (C0 * m) ** 2
    c = 2.0 * b / (C0 * m)
    if math.isinf(phi_uv) and c >= 1.0:
        return math.inf  # the sample process escapes with positive probability

    def inner(p1):
        def f(p2):
            g = a * (1.0 / p2**2 - 1.0 / p1**2) + c * math.log(p2 / p1)
            return math.exp(g) / quad_noise(p2, m) ** 2
        # integrand is largest at p2 = p1 and decays on the scale p1^3 / a
        width = p1**3 / a
        upper = phi_uv
        if math.isinf(upper):
            s1, _ = integrate.quad(f, p1, p1 + 50 * width, limit=200, epsabs=0, epsrel=1e-12)
            s2, _ = integrate.quad(f, p1 + 50 * width, np.inf, limit=200, epsabs=1e-13 * s1,
                                   epsrel=1e-10)
            return s1 + s2
        pts = [x for x in (p1 + width, p1 + 10 * width) if x < upper]
        s, _ = integrate.quad(f, p1, upper, points=pts or None, limit=400, epsabs=0, epsrel=1e-12)
        return s

    with warnings.catch_warnings():
        # the far tail of the inner integral underflows; quad reports that as roundoff
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _ = integrate.quad(lambda p1: 2.0 * inner(p1), phi_end, phi_in, limit=200, epsabs=0,
                                epsrel=1e-10)
    return val


def _grid_operator(x, drift, noise):
    """Second-order FD generator (S^2/2) d2 + (D+B) d on x, Dirichlet at x[0],
    Neumann (mirror) at x[-1]; returns (L, interior diag info)."""
    n = x.size
    h = x[1] - x[0]
    a = noise(x) ** 2 / 2.0
    c = drift(x)
    lo = a / h**2 - c / (2 * h)
    mid = -2 * a / h**2
    up = a / h**2 + c / (2 * h)
    L = sp.lil_matrix((n, n))
    L[0, 0] = 1.0
    for i in range(1, n - 1):
        L[i, i - 1] = lo[i]
        L[i, i] = mid[i]
        L[i, i + 1] = up[i]
    # reflecting wall: ghost node x[n] = x[n-2] (zero derivative)
    L[n - 1, n - 2] = 2 * a[-1] / h**2
    L[n - 1, n - 1] = -2 * a[-1] / h**2
    return L.tocsr()


def backward_moments_fd(phi_in, drift, noise, phi_end, phi_uv, n=20001):
    """(<N>, Var N) at phi_in from the first two backward equations."""
    x = np.linspace(phi_end, phi_uv, n)
    L = _grid_operator(x, drift, noise)
    r1 = -np.ones(n)
    r1[0] = 0.0
    T1 = spla.spsolve(L, r1)
    r2 = -2.0 * T1
    r2[0] = 0.0
    T2 = spla.spsolve(L, r2)
    m1 = float(np.interp(phi_in, x, T1))
    m2 = float(np.interp(phi_in, x, T2))
    return m1, m2 - m1 * m1


def survival_pde(phi_in, drift, noise, phi_end, phi_uv, N_grid, n=4001, dN=2e-3):
    """Q(phi_in, N) for each N in N_grid (increasing), backward Euler."""
    x = np.linspace(phi_end, phi_uv, n)
    h = x[1] - x[0]
    a = noise(x) ** 2 / 2.0
    c = drift(x)
    if np.any(h > 2 * a[1:] / np.maximum(np.abs(c[1:]), 1e-300)):
        raise ValueError("grid too coarse for a monotone central scheme")
    L = _grid_operator(x, drift, noise).tolil()
    L[0, 0] = 0.0  # Q(phi_end) = 0 stays 0 under the update
    L = L.tocsc()
    A = (sp.identity(n, format="csc") - dN * L).tocsc()
    solve = spla.factorized(A)
    Q = np.ones(n)
    Q[0] = 0.0
    out = []
    t = 0.0
    for target in N_grid:
        while t < target - 1e-12:
            Q = solve(Q)
            Q[0] = 0.0
            t += dN
        out.append(float(np.interp(phi_in, x, Q)))
    return np.array(out)


def inverse_gaussian(distance, speed, sigma):
    """Frozen scipy distribution of the first time Brownian motion with drift
    `speed` > 0 toward a barrier at `distance` and volatility `sigma` hits it."""
    mu = distance / speed
    lam = distance**2 / sigma**2
    return stats.invgauss(mu=mu / lam, scale=lam)


def bgk_distance(distance, sigma, dN):
    """Barrier shift for a discretely monitored walk (Broadie–Glasserman–Kou)."""
    return distance + BGK_BETA * sigma * math.sqrt(dN)


def path_log_likelihood_ratio(phi, b_used, drift_fn, noise_fn, dN):
    """ln p_T(X) - ln p_S(X) for a recorded path, from the Gaussian step
    densities of §2.2 Eqs. (13)-(14) evaluated with scipy.stats.norm."""
    x0 = phi[:-1]
    dx = np.diff(phi)
    D = drift_fn(x0)
    S = noise_fn(x0)
    B = b_used * S
    lt = stats.norm.logpdf(dx, loc=D * dN, scale=S * math.sqrt(dN))
    ls = stats.norm.logpdf(dx, loc=(D + B) * dN, scale=S * math.sqrt(dN))
    return float(np.sum(lt - ls))
