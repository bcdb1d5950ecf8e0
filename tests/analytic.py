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
* ``backward_raw_moments``: <N^k>, k = 1..K, from the chain of backward
  equations L T_k = -k T_{k-1} (T_0 = 1) — the moments that Appendix B
  Eq. (B.12) takes from derivatives of the characteristic function at t = 0.
* ``generator_eigenvalues``: the smallest decay rates of the same finite
  difference generator (the poles Lambda_n of Appendix A, Eq. (A.7)).
* ``quad_poles``, ``quad_pole_residues``, ``quad_tail_from_poles``: Appendix A
  for quadratic inflation with a reflecting wall — the pole equation A = B
  (Eq. (A.16)) solved on the negative imaginary t axis, the residues by
  l'Hopital's rule (Eq. (A.18)), and P(N), Q(N) as sums of decaying
  exponentials (Eqs. (A.7), (A.19)); confluent hypergeometric functions from mpmath.
* ``edgeworth_pdf``: Appendix B, Eq. (B.10), with the probabilists' Hermite
  polynomial He_3(x) = x^3 - 3x (Eq. (B.7) prints x^2 - 1).
* ``mgf_cumulants``, ``SaddlepointDensity``: K(s) = ln E[e^{sN}] and its first
  four derivatives from the Riccati form of the backward equation for the
  characteristic function of Appendix A on the real axis, and the density of N
  by the saddle-point approximation (Daniels 1954) — the far tail where the
  Edgeworth series of Appendix B no longer holds.  Pinned by
  ``constant_model_log_mgf`` (Brownian motion with drift, closed form),
  ``quad_log_mgf_appendix_a`` (the hypergeometric solution of Appendix A) and
  the backward cumulants.
* ``em_classical_shift``: the delay of the noise-free Euler-Maruyama map
  against the classical duration (the leading O(dN) bias of <N>).
* ``log_characteristic_function``, ``FourierDensity``: ln E[e^{iwN}] from the
  same Riccati equation at s = i w, and the density by Fourier inversion: the
  bulk and near tail of regimes where the saddle point fails (interim masses,
  where upward excursions make E[e^{sN}] infinite).
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


def backward_raw_moments(phi_in, drift, noise, phi_end, phi_uv, k_max=4, n=20001):
    """[<N>, <N^2>, ..., <N^k_max>] at phi_in: L T_k = -k T_{k-1}, T_0 = 1,
    T_k(phi_end) = 0, T_k'(phi_uv) = 0 (second-order finite differences)."""
    x = np.linspace(phi_end, phi_uv, n)
    solve = spla.factorized(_grid_operator(x, drift, noise).tocsc())
    T = np.ones(n)
    out = []
    for k in range(1, k_max + 1):
        r = -k * T
        r[0] = 0.0
        T = solve(r)
        out.append(float(np.interp(phi_in, x, T)))
    return out


def backward_cumulants(phi_in, drift, noise, phi_end, phi_uv, n=20001):
    """(kappa_1..kappa_4) of N at phi_in.  With chi = exp(K), K = sum kappa_n
    (it)^n / n!, the equation L chi = -it chi (L = a d2 + D d, a = S^2/2: the
    generator of Eq. (A.2)) gives, order by order in it,
        L k1 = -1,  L k2 = -2 a k1'^2,  L k3 = -6 a k1' k2',
        L k4 = -a (6 k2'^2 + 8 k1' k3'),
    with k_n(phi_end) = 0, k_n'(phi_uv) = 0: the cumulants without the
    cancellation of raw moments (Appendix B needs them at a few sigma / <N>)."""
    x = np.linspace(phi_end, phi_uv, n)
    a = noise(x) ** 2 / 2.0
    solve = spla.factorized(_grid_operator(x, drift, noise).tocsc())

    def sol(rhs):
        r = np.array(rhs, dtype=np.float64)
        r[0] = 0.0
        return solve(r)
    d = lambda f: np.gradient(f, x)
    k1 = sol(-np.ones(n))
    d1 = d(k1)
    k2 = sol(-2 * a * d1 ** 2)
    d2 = d(k2)
    k3 = sol(-6 * a * d1 * d2)
    d3 = d(k3)
    k4 = sol(-a * (6 * d2 ** 2 + 8 * d1 * d3))
    return tuple(float(np.interp(phi_in, x, k)) for k in (k1, k2, k3, k4))


def generator_eigenvalues(drift, noise, phi_end, phi_uv, k=3, n=20001):
    """The k smallest decay rates Lambda of L psi = -Lambda psi, psi(phi_end) = 0,
    psi'(phi_uv) = 0 (finite differences, shift-invert about 0)."""
    x = np.linspace(phi_end, phi_uv, n)
    L = _grid_operator(x, drift, noise).tolil()
    L = L[1:, 1:].tocsc()  # eliminate the Dirichlet node
    vals = spla.eigs(L, k=k, sigma=0.0, which="LM", return_eigenvectors=False)
    return np.sort(-vals.real)


# ---- Appendix A: poles and residues for quadratic inflation with a wall ----

def _mp():
    import mpmath  # test-only dependency, available where the CPU tests run
    return mpmath


def _quad_f(mp, m, alpha, phi):
    """f(t, phi) of Eq. (A.11) and df/dphi, with v = m^2 phi^2 / (48 pi^2)
    (the reduced potential V / (24 pi^2) of Eq. (A.3) for V = m^2 phi^2 / 2);
    g is the same with alpha -> -alpha."""
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)
    v = v0 * mp.mpf(phi) ** 2
    a, b = (-1 - alpha) / 4, 1 - alpha / 2
    z = -1 / v
    M = mp.hyp1f1(a, b, z)
    dM = a / b * mp.hyp1f1(a + 1, b + 1, z)  # d/dz 1F1(a; b; z)
    e = (1 + alpha) / 4
    f = v ** e * M
    dfdv = e * v ** (e - 1) * M + v ** e * dM / v ** 2
    return f, dfdv * 2 * v0 * mp.mpf(phi)


def _pole_function(mp, m, phi_end, phi_uv, kappa):
    """On t = -i Lambda with Lambda > v0/4, alpha = i kappa and g = conj(f), so
    A = B (Eq. (A.16)) is the real condition Im[f'(phi_uv) conj(f(phi_end))] = 0."""
    al = 1j * mp.mpf(kappa)
    fe, _ = _quad_f(mp, m, al, phi_end)
    _, fu = _quad_f(mp, m, al, phi_uv)
    return mp.im(fu * mp.conj(fe))


def quad_poles(m, phi_uv, n_poles, phi_end=math.sqrt(2.0), dps=40, dk=0.5):
    """[(Lambda_n, kappa_n)] for n < n_poles: roots kappa > 0 of the pole
    equation (kappa = 0, where f = g and A = B trivially, is no pole), bracketed
    on a grid of step dk and refined; Lambda = v0 (1 + kappa^2) / 4."""
    mp = _mp()
    mp.mp.dps = dps
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)
    F = lambda k: _pole_function(mp, m, phi_end, phi_uv, k)
    out = []
    k0, f0 = dk, F(dk)
    while len(out) < n_poles:
        k1 = k0 + dk
        f1 = F(k1)
        if f0 * f1 < 0:
            r = mp.findroot(F, (k0, k1), solver="anderson")
            out.append((float(v0 * (1 + r * r) / 4), r))
        k0, f0 = k1, f1
    return out


def quad_pole_residues(m, phi_uv, phi, poles, phi_end=math.sqrt(2.0), dps=40):
    """a_n(phi) of Eq. (A.18): -i N(t_n) / D'(t_n) with N = B f/f_end - A g/g_end,
    D = B - A, A = f'_uv / g'_uv, B = f_end / g_end (Eq. (A.14)).  D' is taken
    along kappa (t = -i v0 (1 + kappa^2)/4, dt/dkappa = -i v0 kappa / 2), which
    keeps the derivative off the branch cut of alpha(t)."""
    mp = _mp()
    mp.mp.dps = dps
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)

    def AB(k):
        al = 1j * k
        fe, _ = _quad_f(mp, m, al, phi_end)
        ge, _ = _quad_f(mp, m, -al, phi_end)
        _, fu = _quad_f(mp, m, al, phi_uv)
        _, gu = _quad_f(mp, m, -al, phi_uv)
        return fu / gu, fe / ge, fe, ge

    res = []
    for _, k in poles:
        A, B, fe, ge = AB(k)
        f, _ = _quad_f(mp, m, 1j * k, phi)
        g, _ = _quad_f(mp, m, -1j * k, phi)
        num = B * f / fe - A * g / ge
        dD = mp.diff(lambda kk: AB(kk)[1] - AB(kk)[0], k) / (-1j * v0 * k / 2)
        a = -1j * num / dD
        res.append(float(mp.re(a)))
    return res


def quad_tail_from_poles(m, phi_uv, phi_in, N_values, n_poles=12, phi_end=math.sqrt(2.0)):
    """(P(N), Q(N) = P(N' > N)) at phi_in from the first n_poles terms of Eq. (A.7)."""
    poles = quad_poles(m, phi_uv, n_poles, phi_end)
    a = quad_pole_residues(m, phi_uv, phi_in, poles, phi_end)
    lam = np.array([p[0] for p in poles])
    a = np.array(a)
    N = np.asarray(N_values, dtype=np.float64)[:, None]
    P = np.sum(a * np.exp(-lam * N), axis=1)
    Q = np.sum(a / lam * np.exp(-lam * N), axis=1)
    return P, Q, lam, a


# ---- Appendix B: Edgeworth expansion ----

def hermite_he(k, x):
    """Probabilists' Hermite polynomials He_3, He_4, He_6."""
    if k == 3:
        return x ** 3 - 3 * x
    if k == 4:
        return x ** 4 - 6 * x ** 2 + 3
    if k == 6:
        return x ** 6 - 15 * x ** 4 + 45 * x ** 2 - 15
    raise ValueError(k)


def edgeworth_pdf(x, mu, sigma, gamma, kappa):
    """Eq. (B.10): Gaussian times 1 + gamma/6 He_3 + kappa/24 He_4 + gamma^2/72 He_6."""
    z = (np.asarray(x, dtype=np.float64) - mu) / sigma
    g = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi * sigma * sigma)
    return g * (1 + gamma / 6 * hermite_he(3, z) + kappa / 24 * hermite_he(4, z) + gamma ** 2 / 72 * hermite_he(6, z))


def cumulant_shape(raw):
    """(mu, sigma, gamma, kappa) from raw moments [<N>, <N^2>, <N^3>, <N^4>]."""
    m1, m2, m3, m4 = raw
    var = m2 - m1 ** 2
    c3 = m3 - 3 * m1 * m2 + 2 * m1 ** 3
    c4 = m4 - 4 * m1 * m3 + 6 * m1 ** 2 * m2 - 3 * m1 ** 4
    s = math.sqrt(var)
    return m1, s, c3 / s ** 3, c4 / var ** 2 - 3


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


# ---- the moment generating function of N and its saddle-point inversion ----

def mgf_cumulants(s, phi_in, drift, noise, phi_end, phi_top, rtol=1e-12):
    """(K, K', K'', K''', K'''') at real s, K(s) = ln E[exp(s N)] for runs from
    phi_in: the characteristic function of Appendix A (Eq. (A.2)) on the real
    axis.  M = E[e^{sN}] solves (S^2/2) M'' + D M' + s M = 0 with M(phi_end) = 1
    and M'(phi_top) = 0 (reflecting wall); y = M'/M obeys the Riccati equation
    y' = -y^2 - (2/S^2)(D y + s).  It is stiff when drift dominates (2|D|/S^2 is
    huge) but stable integrated from the wall down to phi_end (Radau).  The
    s-derivatives y_k obey the differentiated equations, and
    K^(k)(s) = integral of y_k from phi_end to phi_in.  Finite for s below the
    domain's leading decay rate."""
    from scipy.integrate import solve_ivp

    def rhs(phi, u):
        y0, y1, y2, y3, y4 = u[:5]
        S = noise(phi)
        g = 2.0 / (S * S)
        D = drift(phi)
        return [-y0 * y0 - g * (D * y0 + s),
                -2 * y0 * y1 - g * (D * y1 + 1.0),
                -2 * y1 * y1 - 2 * y0 * y2 - g * D * y2,
                -6 * y1 * y2 - 2 * y0 * y3 - g * D * y3,
                -6 * y2 * y2 - 8 * y1 * y3 - 2 * y0 * y4 - g * D * y4,
                y0, y1, y2, y3, y4]

    def jac(phi, u):
        y0, y1, y2, y3, y4 = u[:5]
        S = noise(phi)
        c = -2 * y0 - 2.0 * drift(phi) / (S * S)
        J = np.zeros((10, 10))
        J[0, 0] = c
        J[1, 0], J[1, 1] = -2 * y1, c
        J[2, 0], J[2, 1], J[2, 2] = -2 * y2, -4 * y1, c
        J[3, 0], J[3, 1], J[3, 2], J[3, 3] = -2 * y3, -6 * y2, -6 * y1, c
        J[4, 0], J[4, 1], J[4, 2], J[4, 3], J[4, 4] = -2 * y4, -8 * y3, -12 * y2, -8 * y1, c
        J[5:, :5] = np.eye(5)
        return J
    sol = solve_ivp(rhs, (phi_top, phi_end), np.zeros(10), method="Radau", jac=jac, rtol=rtol, atol=1e-14,
                    dense_output=True)
    if not sol.success:
        raise ArithmeticError(f"mgf_cumulants(s = {s}): {sol.message}")
    return tuple(float(v) for v in sol.sol(phi_in)[5:] - sol.y[5:, -1])


class SaddlepointDensity:
    """The density of N from K(s) = ln E[e^{sN}] by the saddle-point
    approximation with its first correction (Daniels 1954):
        f(N) = exp(K(s) - s N) / sqrt(2 pi K''(s)) (1 + lambda_4/8 - 5 lambda_3^2/24),
    K'(s) = N, lambda_k = K^(k)(s) / K''(s)^(k/2).  K, K', K'' and K''' are
    tabulated on a grid of s and interpolated by cubic Hermite polynomials built
    on the exact derivatives (K'''' linearly), so one table serves every N with
    K'(s) inside it."""

    def __init__(self, s_grid, table, mgf=None):
        from scipy.interpolate import CubicHermiteSpline
        self.mgf = mgf
        self.s = np.asarray(s_grid, dtype=np.float64)
        t = np.asarray(table, dtype=np.float64)
        self.t = t
        self.K = CubicHermiteSpline(self.s, t[:, 0], t[:, 1])
        self.K1 = CubicHermiteSpline(self.s, t[:, 1], t[:, 2])
        self.K2 = CubicHermiteSpline(self.s, t[:, 2], t[:, 3])
        self.K3 = CubicHermiteSpline(self.s, t[:, 3], t[:, 4])

    @classmethod
    def from_mgf(cls, s_grid, mgf):
        return cls(s_grid, [mgf(s) for s in s_grid], mgf)

    def saddlepoint(self, N):
        from scipy.optimize import brentq
        return brentq(lambda s: float(self.K1(s)) - N, self.s[0], self.s[-1], xtol=1e-13, rtol=1e-15)

    def pdf(self, N, correction=True, exact=False):
        """exact=True refines each saddle point by Newton steps on the
        generating function itself and takes K and its derivatives from it
        (a few solves per N) instead of the table."""
        out = []
        for x in np.atleast_1d(np.asarray(N, dtype=np.float64)):
            s = self.saddlepoint(x)
            if exact:
                for _ in range(8):  # Newton on K'(s) = N with the exact derivatives
                    k0, k1, k2, k3, k4 = self.mgf(s)
                    if abs(k1 - x) <= 1e-13 * abs(x):
                        break
                    s -= (k1 - x) / k2
            else:
                k0, k2, k3 = float(self.K(s)), float(self.K2(s)), float(self.K3(s))
                k4 = float(np.interp(s, self.s, self.t[:, 4]))
            f = math.exp(k0 - s * x) / math.sqrt(2 * math.pi * k2)
            if correction:
                l3, l4 = k3 / k2 ** 1.5, k4 / k2 ** 2
                f *= 1 + l4 / 8 - 5 * l3 * l3 / 24
            out.append(f)
        return np.array(out)

    def bin_average(self, lo, hi, nodes=6):
        """(1/(hi - lo)) integral of the density over (lo, hi], Gauss-Legendre."""
        x, w = np.polynomial.legendre.leggauss(nodes)
        return 0.5 * float(np.sum(w * self.pdf(0.5 * (hi - lo) * x + 0.5 * (hi + lo))))


def constant_model_log_mgf(s, distance, speed, sigma):
    """ln E[e^{sN}] for Brownian motion with drift `speed` > 0 toward a barrier at
    `distance` and volatility sigma: (distance/sigma^2)(speed - sqrt(speed^2 - 2 sigma^2 s))."""
    return distance / sigma**2 * (speed - math.sqrt(speed * speed - 2 * sigma * sigma * s))


def quad_log_mgf_appendix_a(s, m, phi, phi_end, phi_uv, dps=30):
    """ln E[e^{sN}] for quadratic inflation with a reflecting wall from the
    closed form of Appendix A: chi = (f g'_uv - g f'_uv) / (f_end g'_uv - g_end f'_uv)
    with f, g of Eq. (A.11) at alpha = sqrt(1 - 4 s / v0) (imaginary above
    s = v0/4, where f and g are complex conjugates and chi is real)."""
    mp = _mp()
    mp.mp.dps = dps
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)
    al = mp.sqrt(mp.mpc(1 - 4 * mp.mpf(s) / v0))
    f, _ = _quad_f(mp, m, al, phi)
    g, _ = _quad_f(mp, m, -al, phi)
    fe, _ = _quad_f(mp, m, al, phi_end)
    ge, _ = _quad_f(mp, m, -al, phi_end)
    _, fu = _quad_f(mp, m, al, phi_uv)
    _, gu = _quad_f(mp, m, -al, phi_uv)
    chi = (f * gu - g * fu) / (fe * gu - ge * fu)
    return float(mp.log(mp.re(chi)))


def em_classical_shift(phi_in, dN, phi_end=math.sqrt(2.0)):
    """How much later the noise-free Euler-Maruyama map of quadratic inflation,
    phi <- phi - 2 dN / phi (§2.2 Eq. (11) without noise and bias), crosses
    phi_end than the classical N_cl = (phi_in^2 - phi_end^2)/4, with the
    crossing interpolated linearly within the last step.  To first order in dN
    it is dN/2 ln(phi_in/phi_end): the leading discretisation error of <N> in
    drift domination."""
    phi, k = phi_in, 0
    while True:
        nxt = phi - 2.0 * dN / phi
        if nxt <= phi_end:
            return (k + (phi - phi_end) / (phi - nxt)) * dN - (phi_in ** 2 - phi_end ** 2) / 4.0
        phi, k = nxt, k + 1


def log_characteristic_function(w, phi_in, drift, noise, phi_end, phi_top, rtol=1e-11):
    """ln E[exp(i w N)] for real w: the characteristic function of Appendix A
    (Eq. (A.2)) from the same Riccati equation as mgf_cumulants with s = i w,
    y = u + i v:  u' = -(u^2 - v^2) - (2/S^2) D u,  v' = -2 u v - (2/S^2)(D v + w),
    integrated from the wall down to phi_end (Radau).  Finite for every w,
    unlike the moment generating function, so it also covers regimes where
    excursions towards the wall make E[e^{sN}] diverge."""
    from scipy.integrate import solve_ivp

    def rhs(phi, z):
        u, v = z[0], z[1]
        S = noise(phi)
        g = 2.0 / (S * S)
        D = drift(phi)
        return [-(u * u - v * v) - g * D * u, -2 * u * v - g * (D * v + w), u, v]

    def jac(phi, z):
        u, v = z[0], z[1]
        S = noise(phi)
        c = -2 * u - 2.0 * drift(phi) / (S * S)
        return np.array([[c, 2 * v, 0, 0], [-2 * v, c, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0]])
    sol = solve_ivp(rhs, (phi_top, phi_end), np.zeros(4), method="Radau", jac=jac, rtol=rtol, atol=1e-14,
                    dense_output=True)
    if not sol.success:
        raise ArithmeticError(f"log_characteristic_function(w = {w}): {sol.message}")
    d = sol.sol(phi_in)[2:] - sol.y[2:, -1]
    return complex(d[0], d[1])


class FourierDensity:
    """The density of N by inverting its characteristic function on a grid
    w_k = k dw, k = 0..K: f(N) = (1/pi) sum_k' Re[chi(w_k) e^{-i w_k N}] dw
    (trapezoid, half weight at w = 0).  Exact up to the truncation at K dw
    (where |chi| must be negligible) and to aliasing from N +- 2 pi/dw (where
    the density must be negligible); the absolute accuracy is ~1e-13 of the
    peak, so it serves the bulk and the near tail."""

    def __init__(self, dw, n_w, log_cf):
        self.w = dw * np.arange(n_w)
        self.chi = np.exp(np.array([log_cf(w) for w in self.w]))
        self.wt = np.full(n_w, dw)
        self.wt[0] = 0.5 * dw

    def pdf(self, N):
        N = np.atleast_1d(np.asarray(N, dtype=np.float64))[:, None]
        f = np.real(self.chi[None, :] * np.exp(-1j * self.w[None, :] * N))
        return (f * self.wt).sum(axis=1) / math.pi

    def bin_average(self, lo, hi, nodes=8):
        x, w = np.polynomial.legendre.leggauss(nodes)
        return 0.5 * float(np.sum(w * self.pdf(0.5 * (hi - lo) * x + 0.5 * (hi + lo))))


# ---------------------------------------------------------------------------
# No reflecting wall (phi_uv -> infinity): Appendix A's branch-cut integral
# ---------------------------------------------------------------------------
def no_wall_chi(t, m, phi, phi_end=math.sqrt(2.0), dps=50):
    """chi(t, phi) = E[e^{itN}] without a wall, Appendix A (infinite phi_uv):
    only the g branch of Eq. (A.11) stays bounded as v -> infinity, so
    chi = g(t, phi) / g(t, phi_end), with alpha(t) = sqrt(1 - 4 i t / v0) on the
    principal branch.  t may be complex (an mpmath number or a Python complex)."""
    mp = _mp()
    mp.mp.dps = dps
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)
    al = mp.sqrt(1 - 4j * mp.mpmathify(t) / v0)
    g, _ = _quad_f(mp, m, -al, phi)
    ge, _ = _quad_f(mp, m, -al, phi_end)
    return g / ge


def no_wall_im_chi_on_cut(y, m, phi, phi_end=math.sqrt(2.0), dps=50):
    """Im chi(-i y + 0, phi) for y > v0/4: on the negative imaginary t axis
    approached from Re t > 0, where 1 - 4 i t / v0 = 1 - 4 y / v0 - i 0 and
    alpha = -i kappa, kappa = sqrt(4 y / v0 - 1)."""
    mp = _mp()
    mp.mp.dps = dps
    v0 = mp.mpf(m) ** 2 / (48 * mp.pi ** 2)
    kappa = mp.sqrt(4 * mp.mpf(y) / v0 - 1)
    al = -1j * kappa
    g, _ = _quad_f(mp, m, -al, phi)
    ge, _ = _quad_f(mp, m, -al, phi_end)
    return float(mp.im(g / ge))


def no_wall_branch_cut(m, phi, N_min, phi_end=math.sqrt(2.0), nodes=1600, dps=50, tol=1e-18):
    """The first-passage law without a wall, Appendix A (Eq. (A.28)): closing
    the Fourier inversion P(N) = (1/2pi) int e^{-itN} chi(t) dt (Eq. (A.6))
    around the branch cut of alpha(t) on t = -i y, y > v0/4 (chi has no poles
    there), with chi(-iy - 0) = conj chi(-iy + 0), gives
        P(N) = (1/pi) int_{v0/4}^inf Im chi(-iy + 0, phi) e^{-yN} dy,
        Q(N) = P(N' > N) = (1/pi) int_{v0/4}^inf Im chi(-iy + 0, phi) e^{-yN} / y dy.
    (The printed prefactor, -2 in place of 1/pi, is read as garbled: with it
    the density is neither positive nor normalised.)  With y = v0/4 + s^2 the
    square-root onset at the branch point becomes a smooth integrand, taken by
    Gauss-Legendre on [0, s_max].  |chi| grows along the cut roughly like
    exp(c sqrt(y)), so the Laplace form suits N >= N_min with s_max chosen
    where e^{-y N_min} |Im chi| < tol.  Returns (P, Q) as functions of an
    array of N >= N_min."""
    v0 = m * m / (48.0 * math.pi ** 2)
    y0 = v0 / 4.0
    s_max = 1.0
    while True:
        y = y0 + s_max * s_max
        if abs(no_wall_im_chi_on_cut(y, m, phi, phi_end, dps)) * math.exp(-y * N_min) < tol:
            break
        s_max *= 1.5
    x, w = np.polynomial.legendre.leggauss(nodes)
    s = 0.5 * s_max * (x + 1.0)
    ws = 0.5 * s_max * w * 2.0 * s  # dy = 2 s ds
    y = y0 + s * s
    im = np.array([no_wall_im_chi_on_cut(yy, m, phi, phi_end, dps) for yy in y])

    def P(N):
        N = np.atleast_1d(np.asarray(N, dtype=float))
        return (np.exp(-np.outer(N, y)) * (ws * im)).sum(axis=1) / math.pi

    def Q(N):
        N = np.atleast_1d(np.asarray(N, dtype=float))
        return (np.exp(-np.outer(N, y)) * (ws * im / y)).sum(axis=1) / math.pi

    return P, Q
