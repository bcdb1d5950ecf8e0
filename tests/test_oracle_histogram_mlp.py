"""Pins of the oracle's histogram (brute force with numpy.digitize), its MLP
(torch.nn in float64 on the CPU, autograd, finite differences) and its
tail-objective gradient (finite differences of the brute-force path
log-likelihood ratio).  CPU only."""
import math

import numpy as np
import pytest

import analytic as A
import oracle
from paper_2206_11234_gb300 import workloads as W


def _brute_histogram(N, lw, n_bins, lo, hi, n_sub=1, id_offset=0):
    edges = np.linspace(lo, hi, n_bins + 1)
    fin = np.isfinite(N)
    inside = fin & (N > lo) & (N <= hi)
    j = np.digitize(N, edges, right=True) - 1  # right-closed bins (t_j, t_{j+1}]
    sub = (id_offset + np.arange(N.size)) % n_sub
    out = np.zeros((n_sub, n_bins, 8))
    out[:, :, 0] = -np.inf
    for s in range(n_sub):
        for b in range(n_bins):
            sel = inside & (j == b) & (sub == s)
            if not sel.any():
                continue
            x = lw[sel]
            mx = x.max()
            y = x - mx
            out[s, b] = [mx, np.exp(y).sum(), np.exp(2 * y).sum(), y.sum(), (y ** 2).sum(),
                         (y ** 3).sum(), (y ** 4).sum(), sel.sum()]
    counts = [int((fin & (N <= lo)).sum()), int((fin & (N > hi)).sum()), int((~fin).sum()), N.size]
    return out, np.array(counts)


@pytest.mark.parametrize("n_sub,id_offset", [(1, 0), (3, 5)])
def test_histogram_matches_brute_force(n_sub, id_offset):
    N, lw = W.random_records(5000, seed=3, lo=1.0, hi=4.0)
    got, counts = oracle.histogram(N, lw, 40, 1.0, 4.0, n_sub=n_sub, id_offset=id_offset)
    ref, rc = _brute_histogram(N, lw, 40, 1.0, 4.0, n_sub=n_sub, id_offset=id_offset)
    assert np.array_equal(counts, rc)
    assert np.array_equal(got[..., 7], ref[..., 7])
    assert np.array_equal(got[..., 0], ref[..., 0])
    np.testing.assert_allclose(got[..., 1:7], ref[..., 1:7], rtol=1e-12, atol=1e-9)
    assert got[..., 7].sum() + counts[:3].sum() == N.size
    # the shifted moments give the bin's mean and variance of ln w
    fin = np.isfinite(N) & (N > 1.0) & (N <= 4.0)
    if n_sub == 1:
        b = int(np.argmax(got[0, :, 7]))
        sel = fin & (np.digitize(N, np.linspace(1.0, 4.0, 41), right=True) - 1 == b)
        n = got[0, b, 7]
        assert math.isclose(got[0, b, 0] + got[0, b, 3] / n, lw[sel].mean(), rel_tol=1e-12)
        assert math.isclose((got[0, b, 4] - got[0, b, 3] ** 2 / n) / (n - 1), lw[sel].var(ddof=1),
                            rel_tol=1e-9)


def test_histogram_edge_cases():
    bins, counts = oracle.histogram(np.zeros(0), np.zeros(0), 8, 0.0, 1.0)
    assert counts.tolist() == [0, 0, 0, 0] and np.all(bins[..., 7] == 0)
    assert np.all(bins[..., 0] == -np.inf)
    N = np.array([0.0, 1.0, 1.0 + 1e-15, np.inf, np.nan, -1.0, 0.5])
    lw = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6, -700.0])
    bins, counts = oracle.histogram(N, lw, 2, 0.0, 1.0)
    assert counts.tolist() == [2, 1, 2, 7]
    assert bins[0, 0, 7] == 1 and bins[0, 1, 7] == 1  # 0.5 -> bin 0 (right-closed), 1.0 -> bin 1
    assert bins[0, 0, 0] == -700.0 and bins[0, 0, 1] == 1.0
    # edges that are exact binary fractions: a value on an edge goes to the bin on its left
    e = np.arange(0, 9) / 8.0
    bins, counts = oracle.histogram(e, np.zeros(9), 8, 0.0, 1.0)
    assert counts.tolist() == [1, 0, 0, 9] and np.all(bins[0, :, 7] == 1)
    with pytest.raises(ValueError):
        oracle.histogram(N, lw, 0, 0.0, 1.0)
    with pytest.raises(ValueError):
        oracle.histogram(N, lw, 4, 1.0, 1.0)


def _torch_mlp(params, norm, phi, N):
    torch = pytest.importorskip("torch")
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    H = 64
    W1 = p[: 2 * H].view(H, 2)
    b1 = p[2 * H: 3 * H]
    W2 = p[3 * H: 3 * H + H * H].view(H, H)
    b2 = p[3 * H + H * H: 4 * H + H * H]
    w3 = p[4 * H + H * H: 5 * H + H * H]
    b3 = p[5 * H + H * H]
    x = torch.tensor([(phi - norm[0]) * norm[1], (N - norm[2]) * norm[3]], dtype=torch.float64)
    h1 = torch.tanh(torch.nn.functional.linear(x, W1, b1))
    h2 = torch.tanh(torch.nn.functional.linear(h1, W2, b2))
    out = torch.dot(w3, h2) + b3
    return p, out


def test_mlp_forward_and_backward_match_torch():
    params = W.mlp_params(seed=5, out_scale=1.0)
    norm = (8.0, 0.5, 20.0, 0.05)
    for phi, N in ((8.3, 0.0), (5.1, 17.3), (2.0, 41.0)):
        p, out = _torch_mlp(params, norm, phi, N)
        b, h1, h2 = oracle.mlp_forward(params, norm, phi, N)
        assert abs(b - out.item()) < 1e-13 * (1 + abs(b))
        out.backward()
        g = oracle.mlp_backward(params, norm, phi, N, g=1.0)
        np.testing.assert_allclose(g, p.grad.numpy(), rtol=1e-11, atol=1e-13)
        g2 = oracle.mlp_backward(params, norm, phi, N, g=-2.5)
        np.testing.assert_allclose(g2, -2.5 * g, rtol=1e-13, atol=1e-15)


def test_mlp_backward_matches_finite_differences():
    params = W.mlp_params(seed=9, out_scale=1.0)
    norm = (8.0, 0.5, 20.0, 0.05)
    g = oracle.mlp_backward(params, norm, 7.0, 12.0)
    rng = np.random.default_rng(1)
    for _ in range(5):
        v = rng.normal(size=params.size)
        eps = 1e-6
        fp = oracle.mlp_forward(params + eps * v, norm, 7.0, 12.0)[0]
        fm = oracle.mlp_forward(params - eps * v, norm, 7.0, 12.0)[0]
        assert abs((fp - fm) / (2 * eps) - g @ v) < 1e-7 * (1 + abs(g @ v))


def _mlp_run(params, k_eval=16, **kw):
    args = dict(m=1.0, phi_in=3.0, phi_uv=4.0, dN=1e-3, n_max=3.0, mlp=params,
                mlp_norm=(3.0, 1.0, 1.0, 1.0), k_eval=k_eval)
    args.update(kw)
    return oracle.make_run(**args)


def test_mlp_bias_is_piecewise_constant_and_weight_exact():
    """With the learned bias b is re-evaluated every k_eval steps from the state
    at the block start, and ln w is still the exact path likelihood ratio."""
    params = W.mlp_params(seed=2, out_scale=2.0)
    r = _mlp_run(params)
    D = lambda x: A.quad_drift(x, 0.0, 1.0)
    S = lambda x: A.quad_noise(x, 1.0)
    for i in range(3):
        phi, xi, bu, N, lw = oracle.path(r, i, 100000)
        for k0 in range(0, xi.size, 16):
            ref = oracle.mlp_forward(params, (3.0, 1.0, 1.0, 1.0), phi[k0], k0 * 1e-3)[0]
            assert np.all(bu[k0: k0 + 16] == ref)
        if phi.max() < 4.0:  # no reflection in this path: brute force applies directly
            assert abs(lw - A.path_log_likelihood_ratio(phi, bu, D, S, 1e-3)) < 1e-8 * (1 + abs(lw))


def test_grad_pass_matches_finite_differences_of_path_likelihood():
    """d ln w / d theta at a fixed path (the score used by the tail objective)
    equals the finite difference of the brute-force ln p_T(X) - ln p_S,theta(X)."""
    params = W.mlp_params(seed=4, out_scale=1.0)
    norm = (3.0, 1.0, 1.0, 1.0)
    r = _mlp_run(params, phi_uv=np.inf, n_max=6.0)
    D = lambda x: A.quad_drift(x, 0.0, 1.0)
    S = lambda x: A.quad_noise(x, 1.0)
    i = 2
    coef = np.zeros(i + 1)
    coef[i] = 1.0
    g = oracle.grad_pass(r, coef)
    phi, xi, bu, N, lw = oracle.path(r, i, 100000)

    def llr(p):
        b = np.empty(xi.size)
        for k0 in range(0, xi.size, 16):
            b[k0: k0 + 16] = oracle.mlp_forward(p, norm, phi[k0], k0 * 1e-3)[0]
        return A.path_log_likelihood_ratio(phi, b, D, S, 1e-3)

    rng = np.random.default_rng(3)
    for _ in range(4):
        v = rng.normal(size=params.size)
        eps = 1e-5
        fd = (llr(params + eps * v) - llr(params - eps * v)) / (2 * eps)
        assert abs(fd - g @ v) < 1e-5 * (1 + abs(fd)), (fd, g @ v)
