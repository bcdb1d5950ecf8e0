"""The trained bias network against the zero-variance proposal.

For the tail event E = {N > N*} the proposal whose estimator has zero
variance is the Doob h-transform of the process: its drift is shifted by
S^2 d/dphi ln Q(phi, N* - N), Q the survival function, i.e. in the library's
parametrisation B = b S the amplitude b*(phi, N) = S(phi) d/dphi ln Q(phi, N* - N)
(0 once N > N*).  Q comes from the survival PDE (tests/analytic.py, scipy).
Training minimises the estimator's second moment over the states the
proposal visits, so on the states of the runs that reach the tail — the only
ones the estimator weighs — the trained b must follow b*; elsewhere (near
phi_end, where b* diverges as Q -> 0 and tail runs never go) it is free.

m = 1, phi_in = 8, wall at 9, dN = 5e-4, N* = 40 (the learned-bias workload).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import analytic as A
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SQ2 = math.sqrt(2.0)
M, PHI_IN, UV, DN, TAIL = 1.0, 8.0, 9.0, 5e-4, 40.0


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _bstar_table():
    """d/dphi ln Q(phi, tau) on a grid of phi and tau = 0, 0.25, ..., N*."""
    D, S = (lambda x: A.quad_drift(x, 0.0, M)), (lambda x: A.quad_noise(x, M))
    n, h = 2001, 2e-3
    x = np.linspace(SQ2, UV, n)
    L = A._grid_operator(x, D, S).tolil()
    L[0, 0] = 0.0
    solve = spla.factorized((sp.identity(n, format="csc") - h * L.tocsc()).tocsc())
    Q = np.ones(n)
    Q[0] = 0.0
    taus = np.arange(0.0, TAIL + 1e-9, 0.25)
    field, t = [Q.copy()], 0.0
    for tau in taus[1:]:
        while t < tau - 1e-12:
            Q = solve(Q)
            Q[0] = 0.0
            t += h
        field.append(Q.copy())
    dlnQ = np.gradient(np.log(np.maximum(np.array(field), 1e-300)), x, axis=1)

    def bstar(phi, N):
        it = np.clip(np.rint(np.clip(TAIL - N, 0.0, TAIL) / 0.25).astype(int), 0, len(taus) - 1)
        val = np.array([np.interp(p, x, dlnQ[i]) for p, i in zip(phi, it)])
        return np.where(N < TAIL, S(phi) * val, 0.0)
    return bstar


def test_trained_bias_follows_the_zero_variance_proposal(nat):
    import torch
    base = dict(phi_in=PHI_IN, m=M, dN=DN, n_max=60.0, phi_uv=UV)
    init = W.mlp_params(seed=5, gain=1.0, out_scale=0.05)
    init[-1] = 0.4  # start from the best constant amplitude
    norm = (5.2, 0.5, 30.0, 1.0 / 15.0)
    tr = nat.MlpTrainer(W.SetSpec(n_traj=1 << 15, b=0.0, **base), init, norm, k_eval=64)
    hist = [tr.step(seed=200000 + it, tail_N=TAIL, lr=2e-3) for it in range(160)]
    rel = [h["log_second_moment"] - 2 * math.log(h["p_hat"]) for h in hist]
    assert np.mean(rel[-10:]) < 0.5 * np.mean(rel[:5])
    # the block-start states of fresh runs with the trained network
    nr = 8192
    p = nat.make_params(precision="f32_f64acc", m=M, n_max=60.0, mlp=tr.w, k_eval=64)
    N = torch.empty(nr, dtype=torch.float64, device="cuda")
    lw = torch.empty_like(N)
    rec = torch.empty((int(nr * (60.0 / DN / 64 + 2)), 4), dtype=torch.float32, device="cuda")
    k = nat.fpt_simulate_mlp(p, nat.make_sets([W.SetSpec(n_traj=nr, b=0.0, **base)]), 7, N, lw, rec)
    rec = rec[:k]
    phi0, N0 = rec[:, 0].contiguous(), rec[:, 1].contiguous()
    run = rec[:, 3].contiguous().view(torch.int32).long().cpu().numpy()
    b = torch.empty_like(phi0)
    nat.fpt_mlp_forward(tr.w, phi0, N0, b)
    b = b.cpu().numpy().astype(np.float64)
    bs = _bstar_table()(phi0.cpu().numpy().astype(np.float64), N0.cpu().numpy().astype(np.float64))
    tail_run = (N.cpu().numpy() > TAIL)[run]
    assert tail_run.sum() > 1000
    bb, ss = b[tail_run], bs[tail_run]
    corr = np.corrcoef(bb, ss)[0, 1]
    rms = math.sqrt(np.mean((bb - ss) ** 2))
    print(f"tail-run states: corr(b, b*) {corr:.3f}, rms(b - b*) {rms:.3f}, rms(b*) {math.sqrt(np.mean(ss ** 2)):.3f}, "
          f"relative second moment {rel[0]:.2f} -> {np.mean(rel[-10:]):.2f}")
    assert corr > 0.85, corr
    assert rms < 0.35 * math.sqrt(np.mean(ss ** 2)), rms
