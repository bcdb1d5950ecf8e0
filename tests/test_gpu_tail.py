"""The far tail of the GPU path against the continuum law (quadratic inflation,
m = 1, phi_in = 8, reflecting wall at 9; Appendix A's setting).

The weighted tail P(N > 40) of 2^22 biased runs (b = 0.4, binary32 state,
binary64 log-weight) agrees with the survival PDE, and the decay rate of the
weighted histogram over N in (35, 55] with the leading pole Lambda_0 of the
generator — both computed here with scipy; tests/test_analytic_appendix.py
ties them to the pole expansion of Appendix A (Q(40) = 1.0952e-3,
Lambda_0 = 0.251379).  Tolerances: 4 standard errors plus the O(sqrt(dN))
bias of discretely monitored Euler-Maruyama and the PDE grid error.
"""
import math

import numpy as np
import pytest

import analytic as A
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SQ2 = math.sqrt(2.0)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def test_weighted_tail_and_decay_rate_match_the_continuum(nat):
    import torch
    n = 1 << 22
    spec = W.SetSpec(phi_in=8.0, m=1.0, b=0.4, dN=5e-4, n_max=60.0, n_traj=n, phi_uv=9.0, hist_lo=35.0,
                     hist_hi=55.0, n_bins=20)
    wl = W.Workload("tail", [spec], "f32_f64acc", seed=21)
    N, lw, _, _ = nat.simulate_workload(wl, with_hist=False)
    x = torch.where(N > 40.0, torch.exp(lw), torch.zeros_like(lw))
    est = x.mean().item()
    se = x.std().item() / math.sqrt(n)
    D, S = (lambda z: A.quad_drift(z, 0.0, 1.0)), (lambda z: A.quad_noise(z, 1.0))
    q_pde = A.survival_pde(8.0, D, S, SQ2, 9.0, [40.0], n=4001, dN=2e-3)[0]
    assert abs(est - q_pde) < 4 * se + 5e-3 * q_pde, (est, se, q_pde)
    # decay rate of the weighted density against the generator's leading pole
    bins = nat.empty_bins(spec.n_bins)
    counts = nat.empty_counts(1)
    nat.fpt_histogram(N, lw, spec.n_bins, spec.hist_lo, spec.hist_hi, bins, counts)
    e = nat.empty_estimates(spec.n_bins)
    nat.fpt_estimate(bins, spec.n_bins, spec.hist_lo, spec.hist_hi, n, e)
    g = nat.estimates_to_dict(e)
    mid = spec.hist_lo + (np.arange(spec.n_bins) + 0.5) * (spec.hist_hi - spec.hist_lo) / spec.n_bins
    ok = g["p_direct"] > 0
    y, w = np.log(g["p_direct"][ok]), (g["p_direct"][ok] / g["se_direct"][ok]) ** 2
    slope, _ = np.polyfit(mid[ok], y, 1, w=np.sqrt(w))
    lam0 = A.generator_eigenvalues(D, S, SQ2, 9.0, k=1, n=20001)[0]
    assert abs(-slope / lam0 - 1) < 0.02, (-slope, lam0)
