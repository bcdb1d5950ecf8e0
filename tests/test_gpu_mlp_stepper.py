"""Stepper with the learned bias (tensor-core MLP every k_eval steps).

* Each run's ln w equals the sum over its blocks of -b_k sqrt(dN) Xi_k -
  b_k^2 n_k dN / 2, recomputed from the emitted records with the standalone
  forward kernel (the same b function): the weight of a state-dependent bias
  is booked exactly (§2.2 Eqs. (12)-(14)).
* E[w] = 1 and the weighted first-passage law agrees with the oracle running
  the same bias (FP64 MLP with the same BF16 parameters, same k_eval).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)
NORM = (3.0, 1.0, 2.0, 0.5)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _params():
    p = W.mlp_params(seed=21, gain=1.0, out_scale=0.6)
    p[-1] = 0.5  # b3: a positive bias on average
    return p


def _run(nat, n, seed=0, records=True, k_eval=32, phi_in=3.0, phi_uv=4.0, dN=1e-3, n_max=6.0):
    import torch
    w = nat.mlp_pack(_params(), NORM)
    spec = W.SetSpec(phi_in=phi_in, m=1.0, b=0.0, dN=dN, n_max=n_max, n_traj=n, phi_uv=phi_uv)
    sets = nat.make_sets([spec])
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=n_max, mlp=w, k_eval=k_eval)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    rec = None
    if records:
        cap = int(n * (n_max / dN / k_eval + 2))
        rec = torch.empty((cap, 4), dtype=torch.float32, device="cuda")
    nrec = nat.fpt_simulate_mlp(p, sets, seed, N, lw, rec)
    return w, N, lw, (rec[:nrec] if records else None), nrec


@pytest.mark.parametrize("ks", [16, 32, 64, 128])
def test_log_weight_equals_sum_over_recorded_blocks(nat, ks):
    import torch
    n, dN = 1 << 18, 1e-3  # more runs than resident lanes: refills and parked replays
    w, N, lw, rec, nrec = _run(nat, n, k_eval=ks)
    assert nrec == rec.shape[0] > n
    phi0 = rec[:, 0].contiguous()
    N0 = rec[:, 1].contiguous()
    xi = rec[:, 2].double()
    run = rec[:, 3].contiguous().view(torch.int32).long()
    b = torch.empty_like(phi0)
    nat.fpt_mlp_forward(w, phi0, N0, b)
    b = b.double()
    m0 = torch.round(N0.double() / dN).long()
    # steps of each block: k_eval, except the last block of a run (M - m0)
    Nn = N.clone()
    M = torch.where(torch.isfinite(Nn), torch.ceil(Nn / dN - 1e-9), torch.full_like(Nn, math.ceil(6.0 / dN)))
    last = torch.full((n,), -1, dtype=torch.long, device="cuda").scatter_reduce(0, run, m0, reduce="amax")
    nk = torch.where(m0 == last[run], M.long()[run] - m0, torch.full_like(m0, ks)).double()
    sq = math.sqrt(dN)
    term = -b * sq * xi - 0.5 * b * b * nk * dN
    mag = (b.abs() * sq * xi.abs() + 0.5 * b * b * nk * dN)
    ref = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, run, term)
    scale = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, run, mag)
    err = (lw - ref).abs()
    assert (err <= 1e-4 * (1 + scale)).all(), err.max().item()
    # every run is covered by its blocks: sum of block lengths = M
    cover = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, run, nk)
    assert torch.equal(cover, M)


def test_mean_weight_one_and_agreement_with_oracle(nat):
    import torch
    n = 1 << 16
    w, N, lw, _, _ = _run(nat, n, seed=3, records=False)
    N = N.cpu().numpy()
    lw = lw.cpu().numpy()
    wt = np.exp(lw)
    assert abs(wt.mean() - 1) < 4 * wt.std() / math.sqrt(n)
    # the oracle with the FP64 MLP on the same BF16 parameters, same seeds
    p64 = nat.mlp_unpack_bf16(_params()).numpy()
    m = 2048
    r = oracle.make_run(m=1.0, phi_in=3.0, phi_uv=4.0, dN=1e-3, n_max=6.0, seed=3, mlp=p64, mlp_norm=NORM,
                        k_eval=32)
    No, lo, _ = oracle.simulate(r, m)
    # per run the paths differ only through BF16 rounding of b: same crossing for most runs
    fin = np.isfinite(No) & np.isfinite(N[:m])
    assert np.median(np.abs(N[:m][fin] - No[fin])) < 5e-3
    assert np.median(np.abs(lw[:m] - lo)) < 0.05
    # weighted P(N > t) agree within the combined statistical error
    for t in (1.0, 1.5, 2.0, 3.0):
        a = wt[:m] * (N[:m] > t)
        c = np.exp(lo) * (No > t)
        se = math.hypot(a.std(), c.std()) / math.sqrt(m)
        assert abs(a.mean() - c.mean()) < 4 * se + 1e-4, t


def test_record_capacity_overflow_reported(nat):
    import torch
    w = nat.mlp_pack(_params(), NORM)
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=4096, phi_uv=4.0)
    sets = nat.make_sets([spec])
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=6.0, mlp=w, k_eval=32)
    N = torch.empty(4096, dtype=torch.float64, device="cuda")
    rec = torch.empty((100, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nat.FptError) as ei:
        nat.fpt_simulate_mlp(p, sets, 0, N, N.clone(), rec)
    assert ei.value.code == nat.FPT_ENOMEM
    p.precision = nat.PREC_F64
    with pytest.raises(nat.FptError) as ei:
        nat.fpt_simulate_mlp(p, sets, 0, N, N.clone(), None)
    assert ei.value.code == nat.FPT_EUNSUPPORTED


def test_batch_of_sets_equals_one_call_per_set(nat):
    """Several parameter sets in one learned-bias launch (different phi_in,
    walls, steps and caps) give, run for run, exactly the records of one call
    per set: a run's network input, its noise and its weight depend only on
    the run, whichever runs share its 128-row tile."""
    import torch
    w = nat.mlp_pack(_params(), NORM)
    specs = [W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=3000, phi_uv=4.0, set_id=0),
             W.SetSpec(phi_in=2.2, m=1.0, b=0.0, dN=2e-3, n_max=4.0, n_traj=1000, set_id=1),
             W.SetSpec(phi_in=3.5, m=1.0, b=0.0, dN=1e-3, n_max=3.0, n_traj=777, phi_uv=3.6, set_id=5),
             W.SetSpec(phi_in=1.6, m=1.0, b=0.0, dN=5e-4, n_max=6.0, n_traj=2049, set_id=2)]
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=6.0, mlp=w, k_eval=32)
    n = sum(s.n_traj for s in specs)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty_like(N)
    nat.fpt_simulate_mlp(p, nat.make_sets(specs), 9, N, lw)
    off = 0
    for s in specs:
        N1 = torch.empty(s.n_traj, dtype=torch.float64, device="cuda")
        l1 = torch.empty_like(N1)
        nat.fpt_simulate_mlp(p, nat.make_sets([s]), 9, N1, l1)
        assert torch.equal(N[off:off + s.n_traj], N1), s.set_id
        assert torch.equal(lw[off:off + s.n_traj], l1), s.set_id
        off += s.n_traj
