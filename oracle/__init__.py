"""FP64 CPU oracle of the importance-sampled first-passage-time method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the GPU library never does.
It shares no code with the CUDA path.  Every function follows a passage of
arXiv:2206.11234 (cited in fpt_oracle.c); the Philox4x32-10 generator follows
Salmon et al., SC'11.

Parity status of each function (what pins it is listed in the tests):
  philox4x32_10      pinned: Triton's CPU interpreter Philox, uniformity
  normals4           pinned: normal-distribution KS and moment tests
  simulate           pinned: inverse-Gaussian law (constant model), <N> and
                     Var N from the backward equations, E[w] = 1, log w = 0 at
                     b = 0, the brute-force path likelihood ratio; power-law
                     bias (§3.4 Eq. (26)): p = 1 equals the constant bias,
                     path likelihood ratio for p = 0, 2.5, 3, backward-equation
                     mean with drift D + A phi^3, E[w] = 1, classical duration;
                     polynomial potential (§2.3 Eq. (17)): c2 = m^2/2 equals the
                     quadratic model, backward-equation moments of a quartic and
                     a phi^2 + phi^4 potential, E[w] = 1
  histogram          pinned: brute-force binning with numpy.digitize; moments
                     of ln w - max_lw against numpy mean / var
  estimate (module)  pinned: scipy.stats normaltest / skewtest / kurtosistest;
                     lognormal mean and error-bar coverage on lognormal
                     weights; reduction to the direct estimate at w = 1 with the
                     binomial error; hand-computed jackknife examples
  mlp_forward/back   pinned: torch.nn on CPU in float64, finite differences
  grad_pass          pinned: finite differences of the path log-likelihood
"""
import ctypes
import math
import os
import threading

import numpy as np

from . import build as _build

MODEL_QUADRATIC = 0
MODEL_CONSTANT = 1
MODEL_POLYNOMIAL = 2
POLY_TERMS = 8
BIAS_CONST = 0
BIAS_POWER = 1
BIAS_MLP = 2
MLP_HIDDEN = 64
MLP_NPARAM = 64 * 2 + 64 + 64 * 64 + 64 + 64 + 1


class OracleRun(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("bias_kind", ctypes.c_int32),
        ("m", ctypes.c_double),
        ("a0", ctypes.c_double),
        ("s0", ctypes.c_double),
        ("phi_in", ctypes.c_double),
        ("phi_end", ctypes.c_double),
        ("phi_uv", ctypes.c_double),
        ("dN", ctypes.c_double),
        ("b", ctypes.c_double),
        ("n_max", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("set_id", ctypes.c_uint32),
        ("traj_offset", ctypes.c_uint64),
        ("mlp", ctypes.POINTER(ctypes.c_double)),
        ("mlp_norm", ctypes.c_double * 4),
        ("k_eval", ctypes.c_int32),
        ("bias_p", ctypes.c_double),
        ("poly", ctypes.c_double * 8),
    ]


_lib = None
_keep = []
_lib_lock = threading.Lock()


def lib():
    global _lib
    with _lib_lock:  # callers may be threads: build and load once
        return _lib_locked()


def _lib_locked():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i64, u32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        L.oracle_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.oracle_normals4.argtypes = [u64, u64, u32, u32, P(d)]
        L.oracle_simulate.argtypes = [P(OracleRun), i64, P(d), P(d), P(i64)]
        L.oracle_simulate.restype = ctypes.c_int
        L.oracle_path.argtypes = [P(OracleRun), i64, i64, P(d), P(d), P(d), P(d), P(d)]
        L.oracle_path.restype = i64
        L.oracle_histogram.argtypes = [P(d), P(d), i64, ctypes.c_int32, d, d, ctypes.c_int32, u64,
                                       P(d), P(i64)]
        L.oracle_histogram.restype = ctypes.c_int
        L.oracle_mlp_forward.argtypes = [P(d), P(d), d, d, P(d), P(d)]
        L.oracle_mlp_forward.restype = d
        L.oracle_mlp_backward.argtypes = [P(d), P(d), d, d, d, P(d)]
        L.oracle_grad_pass.argtypes = [P(OracleRun), i64, P(d), P(d)]
        L.oracle_grad_pass.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def make_run(*, model=MODEL_QUADRATIC, m=1.0, a0=0.0, s0=0.0, phi_in, phi_end=math.sqrt(2.0),
             phi_uv=math.inf, dN, b=0.0, n_max, seed=0, set_id=0, traj_offset=0, mlp=None,
             mlp_norm=(0.0, 1.0, 0.0, 1.0), k_eval=1, bias_p=None, poly=None):
    """One parameter set.  b is the amplitude of B = b S(phi), or, with bias_p
    given, of the power law B = b phi^bias_p (§3.4 Eq. (26)).  poly: the
    coefficients c_k of V = sum_k c_k phi^k for model=MODEL_POLYNOMIAL."""
    r = OracleRun()
    r.model, r.m, r.a0, r.s0 = model, m, a0, s0
    r.phi_in, r.phi_end, r.phi_uv = phi_in, phi_end, phi_uv
    r.dN, r.b, r.n_max = dN, b, n_max
    r.seed, r.set_id, r.traj_offset = seed, set_id, traj_offset
    r.bias_kind = BIAS_CONST
    r.mlp_norm = (ctypes.c_double * 4)(*mlp_norm)
    r.k_eval = k_eval
    if poly is not None:
        c = list(poly) + [0.0] * (POLY_TERMS - len(poly))
        r.poly = (ctypes.c_double * POLY_TERMS)(*c[:POLY_TERMS])
    if bias_p is not None:
        r.bias_kind = BIAS_POWER
        r.bias_p = bias_p
    if mlp is not None:
        arr = np.ascontiguousarray(mlp, dtype=np.float64)
        assert arr.size == MLP_NPARAM
        _keep.append(arr)
        r._mlp_ref = arr
        r.mlp = _ptr(arr, ctypes.c_double)
        r.bias_kind = BIAS_MLP
    return r


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                               _ptr(out, ctypes.c_uint32))
    return out


def normals4(seed, traj, set_id, k):
    out = np.zeros(4)
    lib().oracle_normals4(seed, traj, set_id, k, _ptr(out, ctypes.c_double))
    return out


def simulate(run, n):
    """Returns (N, logw, steps) numpy arrays for runs traj_offset .. traj_offset+n-1."""
    N = np.zeros(n)
    lw = np.zeros(n)
    steps = np.zeros(n, dtype=np.int64)
    rc = lib().oracle_simulate(ctypes.byref(run), n, _ptr(N, ctypes.c_double),
                               _ptr(lw, ctypes.c_double), _ptr(steps, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_simulate: invalid argument")
    return N, lw, steps


def path(run, index, max_steps):
    """One recorded run: (phi[0..M], xi[0..M-1], b[0..M-1], N, logw)."""
    phi = np.zeros(max_steps + 1)
    xi = np.zeros(max_steps)
    bu = np.zeros(max_steps)
    N = ctypes.c_double()
    lw = ctypes.c_double()
    M = lib().oracle_path(ctypes.byref(run), index, max_steps, _ptr(phi, ctypes.c_double),
                          _ptr(xi, ctypes.c_double), _ptr(bu, ctypes.c_double), ctypes.byref(N),
                          ctypes.byref(lw))
    if M < 0:
        raise ValueError("oracle_path: invalid argument or run longer than max_steps")
    return phi[: M + 1], xi[:M], bu[:M], N.value, lw.value


def histogram(N, logw, n_bins, lo, hi, n_sub=1, id_offset=0):
    """Returns (bins[n_sub, n_bins, 8], counts[4]); fields max_lw, s1, s2, l1, l2, l3, l4,
    count, where l_k = sum (ln w - max_lw)^k."""
    N = np.ascontiguousarray(N, dtype=np.float64)
    logw = np.ascontiguousarray(logw, dtype=np.float64)
    bins = np.zeros((n_sub, n_bins, 8))
    counts = np.zeros(4, dtype=np.int64)
    rc = lib().oracle_histogram(_ptr(N, ctypes.c_double), _ptr(logw, ctypes.c_double), N.size,
                                n_bins, lo, hi, n_sub, id_offset, _ptr(bins, ctypes.c_double),
                                _ptr(counts, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_histogram: invalid argument")
    return bins, counts


def mlp_forward(params, norm, phi, N):
    p = np.ascontiguousarray(params, dtype=np.float64)
    nm = np.ascontiguousarray(norm, dtype=np.float64)
    h1 = np.zeros(MLP_HIDDEN)
    h2 = np.zeros(MLP_HIDDEN)
    b = lib().oracle_mlp_forward(_ptr(p, ctypes.c_double), _ptr(nm, ctypes.c_double), phi, N,
                                 _ptr(h1, ctypes.c_double), _ptr(h2, ctypes.c_double))
    return b, h1, h2


def mlp_backward(params, norm, phi, N, g=1.0):
    p = np.ascontiguousarray(params, dtype=np.float64)
    nm = np.ascontiguousarray(norm, dtype=np.float64)
    grad = np.zeros(MLP_NPARAM)
    lib().oracle_mlp_backward(_ptr(p, ctypes.c_double), _ptr(nm, ctypes.c_double), phi, N, g,
                              _ptr(grad, ctypes.c_double))
    return grad


def grad_pass(run, coef):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    grad = np.zeros(MLP_NPARAM)
    rc = lib().oracle_grad_pass(ctypes.byref(run), coef.size, _ptr(coef, ctypes.c_double),
                                _ptr(grad, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_grad_pass: invalid argument")
    return grad


def step_cap(n_max, dN):
    """Number of steps after which a run is censored (same rule as the C code)."""
    return int(math.ceil(n_max / dN))
