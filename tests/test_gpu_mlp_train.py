"""Training of the learned bias on the GPU.

* The gradient of one step (device coefficients, records -> rows, tensor-core
  backward) equals the oracle's FP64 backward applied to the same step's
  records with coefficients w_i^2 1{N_i > N*} / sum_j w_j^2 1{N_j > N*}, within
  the BF16 tolerance of the backward kernel.
* A few dozen Adam steps lower the second moment of the tail estimator
  relative to its mean (higher effective sample size per run).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NORM = (3.5, 1.5, 2.5, 0.4)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _init_params(b0, seed=31):
    p = W.mlp_params(seed=seed, gain=1.0, out_scale=0.05)
    p[-1] = b0
    return p


def test_train_step_gradient_matches_oracle(nat):
    import torch
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=1024, phi_uv=4.0)
    tr = nat.MlpTrainer(spec, _init_params(0.6), NORM, k_eval=32)
    p_before = nat.mlp_unpack_bf16(tr.master.cpu()).numpy()
    tail = 2.0
    stats = tr.step(seed=7, tail_N=tail, lr=1e-4)
    n_rec = stats["n_records"]
    assert 0.05 < stats["frac_in_tail"] < 0.95
    grad = tr.grad.cpu().numpy().astype(np.float64)
    rec = tr.records[:n_rec].cpu()
    phi = rec[:, 0].numpy().astype(np.float64)
    Nin = rec[:, 1].numpy().astype(np.float64)
    xi = rec[:, 2].numpy().astype(np.float64)
    run = rec[:, 3].contiguous().view(torch.int32).numpy()
    N = tr.out_N.cpu().numpy()
    lw = tr.out_logw.cpu().numpy()
    E = N > tail
    mx = lw[E].max()
    c = np.where(E, np.exp(2 * (lw - mx)), 0.0)
    c /= c.sum()
    g = c[run] * (-math.sqrt(spec.dN) * xi)
    ref = np.zeros(nat.MLP_NPARAM)
    for r in np.nonzero(g)[0]:
        ref += oracle.mlp_backward(p_before, NORM, phi[r], Nin[r], g[r])
    H = 64
    for name, sl in {"W1": slice(0, 2 * H), "b1": slice(2 * H, 3 * H), "W2": slice(3 * H, 3 * H + H * H),
                     "b2": slice(3 * H + H * H, 4 * H + H * H), "w3": slice(4 * H + H * H, 5 * H + H * H),
                     "b3": slice(5 * H + H * H, None)}.items():
        assert np.linalg.norm(grad[sl] - ref[sl]) <= 0.03 * np.linalg.norm(ref[sl]) + 1e-7, name


def test_training_lowers_relative_second_moment(nat):
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=8.0, n_traj=1 << 14, phi_uv=4.0)
    tr = nat.MlpTrainer(spec, _init_params(0.3), NORM, k_eval=32)
    tail = 4.0
    hist = []
    for it in range(60):
        s = tr.step(seed=1000 + it, tail_N=tail, lr=3e-3)
        if s["p_hat"] > 0:
            # relative second moment L / P^2: 1 + 1/(n_eff per run); lower is better
            hist.append(s["log_second_moment"] - 2 * math.log(s["p_hat"]))
    assert len(hist) > 40
    first, last = np.mean(hist[:8]), np.mean(hist[-8:])
    assert last < first - 0.3, (first, last)
