"""Element-wise parity of the learned-bias kernels with the FP64 oracle.

The tolerance of every element is an error budget built from the
absolute-value chain rule of the network (|W|, |delta|, and each activation
widened by the spread its pre-activation takes under a relative rounding of
every operand): with A_r the per-row rounding magnitudes of db/dtheta and g_r
the row weights, an element may differ by kappa_r sqrt(sum_r (g_r A_r)^2), the
size of independent per-row rounding errors, plus kappa_a sum_r |g_r| T_r for
the relative error of the hardware tanh (T_r its first-order effect; it does
not average out over rows and dominates 1 - h^2 for saturated units), plus
kappa_s |reference|, a systematic relative error.  An element whose reference is well above that budget is one
a wrong sign, a transposed weight block or a dropped (1 - h^2) factor would
move by more than the budget, so the tests also require that a sign error
would be caught on most elements of each weight group, and a transposed W2
block on most of its elements.

* Forward: every output against the oracle's FP64 forward with the same BF16
  parameters, within kappa_f times the absolute-value forward magnitude.
* Backward: every parameter of the batched tensor-core backward against the
  oracle's FP64 backward on the same rows.
* One training step (§2.2 Eqs. (12)-(16), the score of the tail estimator's
  second moment): every parameter of the device gradient against
  ``oracle.grad_pass``, which re-simulates each run in binary64 with the same
  BF16 network and accumulates c_i (-sqrt(dN) Xi_k) db_k/dtheta over its
  blocks, with c_i = w_i^2 1{N_i > N*} / sum_j w_j^2 1{N_j > N*} taken from the
  oracle's own simulation.  N* sits in a gap of the oracle's N values several
  steps wide, so both sides put the same runs in the tail.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H = 64
GROUPS = {"W1": slice(0, 2 * H), "b1": slice(2 * H, 3 * H), "W2": slice(3 * H, 3 * H + H * H),
          "b2": slice(3 * H + H * H, 4 * H + H * H), "w3": slice(4 * H + H * H, 5 * H + H * H),
          "b3": slice(5 * H + H * H, 5 * H + H * H + 1)}
KAPPA_R = 2.0 ** -6   # per-row rounding: 8 BF16 units (2^-9) per term
KAPPA_A = 2.0 ** -8   # activation as used: BF16 storage (2^-9) and tanh.approx (2^-11), doubled
KAPPA_S = 2.0 ** -7   # systematic relative error
KAPPA_F = 2.0 ** -6   # forward rounding


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _layers(p):
    W1 = p[GROUPS["W1"]].reshape(H, 2)
    W2 = p[GROUPS["W2"]].reshape(H, H)
    return W1, p[GROUPS["b1"]], W2, p[GROUPS["b2"]], p[GROUPS["w3"]], p[GROUPS["b3"]][0]


def _chain(p, norm, phi, N):
    """Per row, two kinds of magnitude of the network's intermediate values.

    Rounding (BF16 operands, FP32 accumulation): activations widened by their
    rounding spread (H1, H2) and the backward deltas (D1, D2) as the exact
    value plus the root-sum-square of the rounded products that make them up;
    these errors are independent from row to row.

    Activation approximation: the first-order change of each value when every
    tanh output carries a relative error (a1, a2 for h1, h2; T1, T2 for the
    deltas through 1 - h^2).  The errors of different units combine as a
    root-sum-square; the error is a fixed function of the pre-activation, so
    over rows it does not average out (summed linearly by grad_budget), and it
    dominates 1 - h^2 for saturated units."""
    W1, b1, W2, b2, w3, _ = _layers(p)
    x = np.stack([(np.asarray(phi, float) - norm[0]) * norm[1], (np.asarray(N, float) - norm[2]) * norm[3]], 1)
    h1 = np.tanh(x @ W1.T + b1)
    t1 = 1 - h1 ** 2
    s1 = t1 * np.sqrt(x ** 2 @ (W1 ** 2).T + b1 ** 2)
    H1 = np.abs(h1) + s1
    h2 = np.tanh(h1 @ W2.T + b2)
    t2 = 1 - h2 ** 2
    s2 = t2 * np.sqrt(H1 ** 2 @ (W2 ** 2).T + b2 ** 2)
    H2 = np.abs(h2) + s2
    D2 = np.abs(w3) * (t2 + 2 * np.abs(h2) * s2)
    e1 = (w3 * t2) @ W2
    D1 = (np.abs(e1) + np.sqrt(D2 ** 2 @ W2 ** 2)) * (t1 + 2 * np.abs(h1) * s1)
    a1 = np.abs(h1)
    a2 = np.abs(h2) + t2 * np.sqrt(a1 ** 2 @ (W2 ** 2).T)
    T2 = np.abs(w3) * 2 * np.abs(h2) * a2
    T1 = np.sqrt(T2 ** 2 @ W2 ** 2) * t1 + np.abs(e1) * 2 * np.abs(h1) * a1
    return dict(x=x, H1=H1, H2=H2, D1=D1, D2=D2, a1=a1, a2=a2, T1=T1, T2=T2, d2=np.abs(w3 * t2))


def forward_magnitude(p, norm, phi, N):
    """Per row: (rounding) root-sum-square of w3_n H2_n plus |b3|, and
    (activation) sum_n |w3_n| a2_n."""
    _, _, _, _, w3, b3 = _layers(p)
    c = _chain(p, norm, phi, N)
    return np.sqrt(c["H2"] ** 2 @ w3 ** 2) + abs(b3), c["a2"] @ np.abs(w3)


def grad_budget(p, norm, phi, N, g):
    """Per parameter: R = sqrt(sum_r (g_r A_r)^2) with A_r the rounding
    magnitude of db/dtheta at row r, and L = sum_r |g_r| T_r with T_r its
    activation-approximation magnitude."""
    c = _chain(p, norm, phi, N)
    x, H1, H2, D1, D2 = c["x"], c["H1"], c["H2"], c["D1"], c["D2"]
    g = np.asarray(g, float)
    g2, ga = g ** 2, np.abs(g)
    R = np.zeros(oracle.MLP_NPARAM)
    R[GROUPS["W1"]] = ((g2[:, None] * D1 ** 2).T @ x ** 2).ravel()
    R[GROUPS["b1"]] = g2 @ D1 ** 2
    R[GROUPS["W2"]] = ((g2[:, None] * D2 ** 2).T @ H1 ** 2).ravel()
    R[GROUPS["b2"]] = g2 @ D2 ** 2
    R[GROUPS["w3"]] = g2 @ H2 ** 2
    R[GROUPS["b3"]] = g2.sum()
    L = np.zeros(oracle.MLP_NPARAM)
    L[GROUPS["W1"]] = ((ga[:, None] * c["T1"]).T @ np.abs(x)).ravel()
    L[GROUPS["b1"]] = ga @ c["T1"]
    L[GROUPS["W2"]] = ((ga[:, None] * c["T2"]).T @ np.abs(c["a1"]) + (ga[:, None] * c["d2"]).T @ c["a1"]).ravel()
    L[GROUPS["b2"]] = ga @ c["T2"]
    L[GROUPS["w3"]] = ga @ c["a2"]
    return np.sqrt(R), L


def _check_elementwise(got, ref, budget_terms, what, teeth=True):
    """|got - ref| <= kappa_r R + kappa_a L + kappa_s |ref| element by element;
    with teeth, a sign error (|got - ref| = 2 |ref|) would exceed the budget on
    most elements of each weight group, and so would a transposed W2 block."""
    R, L = budget_terms
    budget = KAPPA_R * R + KAPPA_A * L + KAPPA_S * np.abs(ref) + 1e-12 * np.max(np.abs(ref))
    ratio = np.abs(got - ref) / budget
    for name, sl in GROUPS.items():
        t = np.abs(ref[sl]) / budget[sl]
        print(f"{what} {name}: max |d|/budget {ratio[sl].max():.3f}, median {np.median(ratio[sl]):.3f}; "
              f"|ref|/budget median {np.median(t):.1f}, sign error caught on {np.mean(2 * t > 1):.2f}")
    worst = int(np.argmax(ratio))
    assert ratio.max() <= 1.0, (what, worst, got[worst], ref[worst], budget[worst])
    if teeth:
        for name, sl in GROUPS.items():
            if sl.stop - sl.start > 1:
                assert np.mean(2 * np.abs(ref[sl]) > budget[sl]) > 0.5, (what, name)
        wt = ref.copy()
        wt[GROUPS["W2"]] = ref[GROUPS["W2"]].reshape(H, H).T.ravel()
        assert np.mean(np.abs(wt - ref)[GROUPS["W2"]] > budget[GROUPS["W2"]]) > 0.5, what


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(1.4, 9.0, n).astype(np.float32)
    N = rng.uniform(0.0, 60.0, n).astype(np.float32)
    g = rng.normal(0.0, 1.0, n).astype(np.float32)
    return phi, N, g


@pytest.mark.parametrize("n", [1, 127, 129, 1000, 20000])
def test_forward_every_output(nat, n):
    import torch
    norm = (5.0, 0.35, 30.0, 1.0 / 30.0)
    params = W.mlp_params(seed=11, gain=1.5, out_scale=1.0)
    w = nat.mlp_pack(params, norm)
    p64 = nat.mlp_unpack_bf16(params).numpy()
    phi, N, _ = _inputs(n, seed=n)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    nat.fpt_mlp_forward(w, torch.from_numpy(phi).cuda(), torch.from_numpy(N).cuda(), out)
    got = out.cpu().numpy().astype(np.float64)
    ref = np.array([oracle.mlp_forward(p64, norm, float(phi[i]), float(N[i]))[0] for i in range(n)])
    F, Fa = forward_magnitude(p64, norm, phi.astype(float), N.astype(float))
    ratio = np.abs(got - ref) / (KAPPA_F * F + KAPPA_A * Fa)
    print(f"forward n = {n}: max |d|/(kappa_f F) {ratio.max():.3f}, median {np.median(ratio):.3f}")
    assert ratio.max() <= 1.0, int(np.argmax(ratio))


@pytest.mark.parametrize("n,positive", [(1, False), (130, False), (2000, False), (2000, True)])
def test_backward_every_parameter(nat, n, positive):
    import torch
    norm = (5.0, 0.35, 30.0, 1.0 / 30.0)
    params = W.mlp_params(seed=12, gain=1.5, out_scale=1.0)
    w = nat.mlp_pack(params, norm)
    p64 = nat.mlp_unpack_bf16(params).numpy()
    phi, N, g = _inputs(n, seed=100 + n)
    if positive:
        g = np.abs(g)
    grad = torch.zeros(nat.MLP_NPARAM, dtype=torch.float32, device="cuda")
    nat.fpt_mlp_backward(w, torch.from_numpy(phi).cuda(), torch.from_numpy(N).cuda(), torch.from_numpy(g).cuda(),
                         grad)
    got = grad.cpu().numpy().astype(np.float64)
    ref = np.zeros(nat.MLP_NPARAM)
    for i in range(n):
        ref += oracle.mlp_backward(p64, norm, float(phi[i]), float(N[i]), float(g[i]))
    B = grad_budget(p64, norm, phi.astype(float), N.astype(float), g.astype(float))
    _check_elementwise(got, ref, B, f"backward n = {n}")


def _gap_threshold(N, dN, lo_q=0.4, hi_q=0.85, min_gap_steps=6):
    """Midpoint of the widest gap between consecutive finite N values in the
    quantile range, if it is at least min_gap_steps steps wide."""
    f = np.sort(N[np.isfinite(N)])
    a, b = int(lo_q * f.size), int(hi_q * f.size)
    gaps = f[a + 1:b] - f[a:b - 1]
    k = int(np.argmax(gaps))
    assert gaps[k] >= min_gap_steps * dN, gaps[k]
    return 0.5 * (f[a + k] + f[a + k + 1])


def test_train_step_gradient_every_parameter_vs_oracle_grad_pass(nat):
    import torch
    norm = (3.5, 1.5, 2.5, 0.4)
    dN, k_eval, seed, n = 1e-3, 32, 7, 1024
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=dN, n_max=6.0, n_traj=n, phi_uv=4.0)
    init = W.mlp_params(seed=31, gain=1.0, out_scale=0.05)
    init[-1] = 0.6
    p64 = nat.mlp_unpack_bf16(torch.as_tensor(init, dtype=torch.float32)).numpy()
    # the oracle's own simulation with the same BF16 network: tail threshold and coefficients
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=dN, n_max=6.0, seed=seed, mlp=p64, mlp_norm=norm,
                        k_eval=k_eval)
    No, lwo, _ = oracle.simulate(r, n)
    tail = _gap_threshold(No, dN)
    E = No > tail
    c = np.where(E, np.exp(2 * (lwo - lwo[E].max())), 0.0)
    c /= c.sum()
    ref = oracle.grad_pass(r, c)
    # the budget: every block of every tail run, from the oracle's recorded paths
    cap = oracle.step_cap(6.0, dN) + 1
    rows_phi, rows_N, rows_g = [], [], []
    for i in np.nonzero(E)[0]:
        phi, xi, _, _, _ = oracle.path(r, int(i), cap)
        for k0 in range(0, xi.size, k_eval):
            rows_phi.append(phi[k0])
            rows_N.append(k0 * dN)
            rows_g.append(c[i] * math.sqrt(dN) * xi[k0:k0 + k_eval].sum())
    B = grad_budget(p64, norm, np.array(rows_phi), np.array(rows_N), np.array(rows_g))
    # the device step: simulate, coefficients, rows, tensor-core backward
    tr = nat.MlpTrainer(spec, init, norm, k_eval=k_eval)
    stats = tr.step(seed=seed, tail_N=tail, lr=1e-4)
    gN = tr.out_N.cpu().numpy()
    assert np.array_equal(gN > tail, E), int(np.sum((gN > tail) != E))
    assert 0.05 < stats["frac_in_tail"] < 0.95
    got = tr.grad.cpu().numpy().astype(np.float64)
    _check_elementwise(got, ref, B, "train step")


def per_bin_z(Na, lwa, Nb, lwb, edges, min_count=400):
    """z = (P_a - P_b) / sqrt(se_a^2 + se_b^2) of the weighted estimates of
    P(N in bin) (§2.1 Eq. (9) with the weights of §2.2 Eq. (16)) over the bins
    where both samples hold at least min_count runs."""
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        est = []
        for N, lw in ((Na, lwa), (Nb, lwb)):
            x = np.where((N > lo) & (N <= hi), np.exp(lw), 0.0)
            est.append((x.mean(), x.std() / math.sqrt(x.size), int(np.count_nonzero(x))))
        (pa, sa, ca), (pb, sb, cb) = est
        if min(ca, cb) >= min_count:
            out.append((pa - pb) / math.hypot(sa, sb))
    return np.array(out)


def assert_bins_agree(z, what):
    """Every bin within 3 combined sigma, read as: the count beyond 3 sigma at
    most the 99.9 % binomial quantile for p = 0.0027, and none beyond 5 sigma."""
    from scipy.stats import binom
    allowed = int(binom.ppf(0.999, z.size, 0.0027))
    print(f"{what}: {z.size} bins, max |z| {np.abs(z).max():.2f}, beyond 3 sigma {int(np.sum(np.abs(z) > 3))} "
          f"(allowed {allowed})")
    assert z.size >= 10, what
    assert np.sum(np.abs(z) > 3) <= allowed and np.abs(z).max() < 5, what


def test_learned_bias_histogram_every_bin_vs_oracle(nat):
    """The learned-bias stepper (tensor-core MLP every 32 steps) against the
    oracle running the same BF16 network in binary64 on other runs: the
    weighted P(N) agrees bin by bin (0.1-wide bins on (0, 6])."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    norm = (3.0, 1.0, 2.0, 0.5)
    params = W.mlp_params(seed=21, gain=1.0, out_scale=0.6)
    params[-1] = 0.5
    w = nat.mlp_pack(params, norm)
    n = 1 << 18
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=n, phi_uv=4.0)
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=6.0, mlp=w, k_eval=32)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    nat.fpt_simulate_mlp(p, nat.make_sets([spec]), 5, N, lw)
    p64 = nat.mlp_unpack_bf16(params).numpy()
    m, chunk = 1 << 17, 1 << 13

    def part(k):
        r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=1e-3, n_max=6.0, seed=6, traj_offset=k * chunk,
                            mlp=p64, mlp_norm=norm, k_eval=32)
        return oracle.simulate(r, chunk)[:2]
    with ThreadPoolExecutor(16) as ex:
        res = list(ex.map(part, range(m // chunk)))
    No = np.concatenate([a for a, _ in res])
    lo = np.concatenate([b for _, b in res])
    z = per_bin_z(N.cpu().numpy(), lw.cpu().numpy(), No, lo, np.linspace(0.0, 6.0, 61))
    assert_bins_agree(z, "learned bias, m = 1, phi_in = 3, wall 4")
