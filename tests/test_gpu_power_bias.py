"""Power-law bias B = A_p phi^p (§3.4 Eq. (26)) on the GPU against the FP64
oracle running the same bias.

* FP64 stepper, per run: the same crossing step for every run, |dN| <= 1e-12 N
  and |d ln w| <= 1e-12 max(1, sum_m |increment_m|), for integer and real p,
  with and without the reflecting wall.
* Binary32 modes: statistical parity (histogram bins within 3 combined sigma,
  <N> and E[w]) and per-run closeness to FP64, for the specialised integer
  powers and the general-p kernel.
* p = 1 with A_1 = b c0 m is the constant bias B = b S.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)
C0 = 1.0 / (2.0 * math.pi * math.sqrt(6.0))


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def gpu_run(nat, *, n, phi_in, dN, amp, p, n_max, m=1.0, phi_uv=math.inf, seed=0, precision="f64"):
    import torch
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    prm = nat.make_params(precision=precision, m=m, n_max=n_max, bias_p=p, steps_out=steps)
    nat.fpt_simulate(prm, n, phi_in, SQ2, phi_uv, dN, amp, seed, N, lw)
    torch.cuda.synchronize()
    return N.cpu().numpy(), lw.cpu().numpy(), int(steps.item())


def oracle_run(*, n, phi_in, dN, amp, p, n_max, m=1.0, phi_uv=math.inf, seed=0):
    r = oracle.make_run(m=m, phi_in=phi_in, phi_uv=phi_uv, dN=dN, b=amp, n_max=n_max, seed=seed, bias_p=p)
    return oracle.simulate(r, n)


CASES = [dict(n=2000, phi_in=3.0, dN=1e-3, amp=0.004, p=3.0, n_max=20.0, phi_uv=4.0),
         dict(n=2000, phi_in=3.0, dN=1e-3, amp=0.01, p=2.5, n_max=20.0, phi_uv=4.0),
         dict(n=2000, phi_in=3.0, dN=1e-3, amp=0.3, p=0.0, n_max=6.0),
         dict(n=600, phi_in=6.0, dN=1e-3, amp=1e-4, p=3.0, n_max=10.0, m=0.01)]


@pytest.mark.parametrize("case", CASES, ids=["p3_wall", "p2.5_wall", "p0", "p3_drift"])
def test_f64_per_run_parity(nat, case):
    N_g, lw_g, st_g = gpu_run(nat, **case)
    N_o, lw_o, st_o = oracle_run(**case)
    assert st_g == int(st_o.sum())
    assert np.array_equal(np.isinf(N_g), np.isinf(N_o))
    fin = np.isfinite(N_o)
    assert np.all(np.abs(N_g[fin] - N_o[fin]) <= 1e-12 * np.maximum(N_o[fin], 1e-300))
    # per-step |increment| <= beta sqrt(dN) |xi| + beta^2 dN / 2 with beta = A phi^(p-1) / (c0 m): bound
    # the sum by the largest beta on the path's range times the step count
    phis = np.array([case["phi_in"], case.get("phi_uv", case["phi_in"]), SQ2])
    phis = phis[np.isfinite(phis)]
    beta = case["amp"] * np.max(phis ** (case["p"] - 1)) / (C0 * case.get("m", 1.0))
    scale = np.maximum(1.0, st_o * (beta * math.sqrt(case["dN"]) * 3.0 + 0.5 * beta * beta * case["dN"]))
    assert np.all(np.abs(lw_g - lw_o) <= 1e-12 * scale), np.max(np.abs(lw_g - lw_o) / scale)


@pytest.mark.parametrize("precision", ["f32_kahan", "f32_f64acc"])
@pytest.mark.parametrize("p", [0.0, 1.0, 2.0, 3.0, 4.0, 2.5])
def test_f32_matches_f64_and_oracle_statistics(nat, precision, p):
    """Every binary32 kernel (p = 0..4 specialised, 2.5 general) against the
    binary64 GPU path on the same runs, and E[w] = 1."""
    amp = {0.0: 0.3, 1.0: 0.8 * C0, 2.0: 0.02, 3.0: 0.004, 4.0: 0.001, 2.5: 0.01}[p]
    case = dict(n=8192, phi_in=3.0, dN=1e-3, amp=amp, p=p, n_max=20.0, phi_uv=4.0)
    N32, lw32, _ = gpu_run(nat, precision=precision, **case)
    N64, lw64, _ = gpu_run(nat, precision="f64", **case)
    fin = np.isfinite(N64) & np.isfinite(N32)
    assert fin.mean() > 0.999
    same = np.abs(N32[fin] - N64[fin]) < case["dN"]
    assert same.mean() > 0.97
    assert np.median(np.abs(N32[fin] - N64[fin])) < 1e-4
    assert np.median(np.abs(lw32 - lw64)) < 1e-4
    assert abs(N32[fin].mean() / N64[fin].mean() - 1) < 2e-3
    w = np.exp(lw32)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(w.size)
    # weighted histograms of the two precisions agree bin by bin
    from oracle import estimate as OE
    a = OE.estimate(N32, lw32, 40, 0.0, 8.0)
    c = OE.estimate(N64, lw64, 40, 0.0, 8.0)
    sig = np.hypot(a["se_direct"], c["se_direct"])
    ok = (np.abs(a["p_direct"] - c["p_direct"]) <= 3 * sig) | (sig == 0)
    assert ok.mean() >= 0.97


def test_p1_is_the_constant_bias(nat):
    import torch
    n, dN, b = 4096, 1e-3, 0.8
    N1, lw1, _ = gpu_run(nat, n=n, phi_in=3.0, dN=dN, amp=b * C0, p=1.0, n_max=6.0, phi_uv=3.5)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    prm = nat.make_params(precision="f64", m=1.0, n_max=6.0)
    nat.fpt_simulate(prm, n, 3.0, SQ2, 3.5, dN, b, 0, N, lw)
    N0, lw0 = N.cpu().numpy(), lw.cpu().numpy()
    fin = np.isfinite(N0)
    assert np.array_equal(fin, np.isfinite(N1))
    np.testing.assert_allclose(N1[fin], N0[fin], rtol=1e-12)
    np.testing.assert_allclose(lw1, lw0, rtol=0, atol=1e-10)


def test_power_bias_in_batches_and_plans(nat):
    """Several amplitudes in one batched launch equal one call each."""
    import torch
    specs = [W.SetSpec(phi_in=6.0, m=0.01, b=a, dN=1e-3, n_max=10.0, n_traj=3000, set_id=i, hist_lo=8.4,
                       hist_hi=9.0, n_bins=60) for i, a in enumerate((0.0, 5e-5, 1e-4))]
    sets = nat.make_sets(specs)
    n = sum(s.n_traj for s in specs)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    bins = nat.empty_bins(180)
    counts = nat.empty_counts(3)
    p = nat.make_params(precision="f32_f64acc", m=0.01, n_max=10.0, bias_p=3.0)
    nat.fpt_simulate_batch(p, sets, 9, N, lw, bins, counts)
    off = 0
    for s in specs:
        Ni = torch.empty(s.n_traj, dtype=torch.float64, device="cuda")
        li = torch.empty_like(Ni)
        q = nat.make_params(precision="f32_f64acc", m=0.01, n_max=10.0, bias_p=3.0, set_id=s.set_id)
        nat.fpt_simulate(q, s.n_traj, s.phi_in, SQ2, math.inf, s.dN, s.b, 9, Ni, li)
        assert torch.equal(Ni, N[off: off + s.n_traj]) and torch.equal(li, lw[off: off + s.n_traj])
        off += s.n_traj
    plan = nat.Plan(p, sets, N, lw, bins, counts)
    N_b = N.clone()
    plan.launch(9)
    assert torch.equal(N, N_b)
    plan.close()


def test_power_bias_argument_checks(nat):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    for kw in (dict(bias_p=math.nan), dict(bias_p=math.inf), dict(bias_p=100.0)):
        p = nat.make_params(precision="f32_kahan", m=1.0, n_max=6.0, **kw)
        with pytest.raises(nat.FptError) as ei:
            nat.fpt_simulate(p, 8, 3.0, SQ2, math.inf, 1e-3, 0.1, 0, x, x.clone())
        assert ei.value.code == nat.FPT_EINVAL
    p = nat.make_params(precision="f32_kahan", m=1.0, n_max=6.0, bias_p=3.0, k_steps=16)
    with pytest.raises(nat.FptError) as ei:
        nat.fpt_simulate(p, 8, 3.0, SQ2, math.inf, 1e-3, 0.1, 0, x, x.clone())
    assert ei.value.code == nat.FPT_EINVAL
    p = nat.make_params(model=nat.MODEL_CONSTANT, precision="f64", s0=1.0, a0=-1.0, n_max=6.0, bias_p=1.0)
    with pytest.raises(nat.FptError) as ei:
        nat.fpt_simulate(p, 8, 2.0, 1.0, math.inf, 1e-3, 0.1, 0, x, x.clone())
    assert ei.value.code == nat.FPT_EUNSUPPORTED
