"""General potential V(phi) = sum_k c_k phi^k (§2.3 Eq. (17)) on the GPU path
against the FP64 oracle running the same potential.

* FP64 stepper, per run: same crossing step, |dN| <= 1e-12 N and
  |d ln w| <= 1e-12 max(1, sum_m |increment_m|) (constant bias B = b S).
* Binary32 modes: per-run closeness to FP64 and E[w] = 1.
* c_2 = m^2 / 2 alone is the quadratic model.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CASES = [dict(c=[0, 0, 0, 0, 0.25 * 0.05], phi_in=4.0, phi_end=math.sqrt(8.0), phi_uv=4.6, b=0.8, n=2000),
         dict(c=[0, 0, 0.5 * 0.3, 0, 0.25 * 0.02], phi_in=3.5, phi_end=1.6, phi_uv=math.inf, b=0.5, n=2000),
         dict(c=[0.02, 0, 0.1, 0.01], phi_in=3.0, phi_end=1.2, phi_uv=3.4, b=0.0, n=2000)]
IDS = ["quartic_wall", "phi2_phi4", "cubic_offset_wall"]


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def gpu_run(nat, case, precision="f64", n_max=40.0, dN=1e-3, seed=0):
    import torch
    n = case["n"]
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = nat.make_params(model=nat.MODEL_POLYNOMIAL, precision=precision, poly=case["c"], n_max=n_max, steps_out=steps)
    nat.fpt_simulate(p, n, case["phi_in"], case["phi_end"], case["phi_uv"], dN, case["b"], seed, N, lw)
    torch.cuda.synchronize()
    return N.cpu().numpy(), lw.cpu().numpy(), int(steps.item())


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_f64_per_run_parity(nat, case):
    N_g, lw_g, st_g = gpu_run(nat, case)
    r = oracle.make_run(model=oracle.MODEL_POLYNOMIAL, poly=case["c"], phi_in=case["phi_in"], phi_end=case["phi_end"],
                        phi_uv=case["phi_uv"], dN=1e-3, b=case["b"], n_max=40.0)
    N_o, lw_o, st_o = oracle.simulate(r, case["n"])
    assert st_g == int(st_o.sum())
    assert np.array_equal(np.isinf(N_g), np.isinf(N_o))
    fin = np.isfinite(N_o)
    assert np.all(np.abs(N_g[fin] - N_o[fin]) <= 1e-12 * N_o[fin])
    b = case["b"]
    scale = np.maximum(1.0, st_o * (abs(b) * math.sqrt(1e-3) * 3.0 + 0.5 * b * b * 1e-3))
    assert np.all(np.abs(lw_g - lw_o) <= 1e-12 * scale)


@pytest.mark.parametrize("precision", ["f32_kahan", "f32_f64acc"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_f32_matches_f64(nat, case, precision):
    c = dict(case, n=8192)
    N32, lw32, _ = gpu_run(nat, c, precision=precision)
    N64, lw64, _ = gpu_run(nat, c)
    fin = np.isfinite(N32) & np.isfinite(N64)
    assert fin.mean() > 0.999
    assert np.mean(np.abs(N32[fin] - N64[fin]) < 1e-3) > 0.97
    assert np.median(np.abs(N32[fin] - N64[fin])) < 1e-4
    assert abs(N32[fin].mean() / N64[fin].mean() - 1) < 2e-3
    assert np.median(np.abs(lw32 - lw64)) < 1e-4 * max(1.0, c["b"])
    w = np.exp(lw32)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(w.size) + 1e-12


def test_quadratic_through_the_polynomial_model(nat):
    import torch
    m, n = 0.7, 3000
    case = dict(c=[0, 0, 0.5 * m * m], phi_in=3.0, phi_end=math.sqrt(2.0), phi_uv=3.5, b=0.7, n=n)
    N1, lw1, _ = gpu_run(nat, case, n_max=6.0)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    p = nat.make_params(precision="f64", m=m, n_max=6.0)
    nat.fpt_simulate(p, n, 3.0, math.sqrt(2.0), 3.5, 1e-3, 0.7, 0, N, lw)
    N0, lw0 = N.cpu().numpy(), lw.cpu().numpy()
    fin = np.isfinite(N0)
    assert np.array_equal(fin, np.isfinite(N1))
    np.testing.assert_allclose(N1[fin], N0[fin], rtol=1e-12)
    np.testing.assert_allclose(lw1, lw0, rtol=0, atol=1e-10)


def test_polynomial_argument_checks(nat):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = nat.make_params(model=nat.MODEL_POLYNOMIAL, precision="f32_kahan", poly=[0, 0, 0.1], n_max=6.0, bias_p=3.0)
    with pytest.raises(nat.FptError) as ei:
        nat.fpt_simulate(p, 8, 3.0, 1.0, math.inf, 1e-3, 0.1, 0, x, x.clone())
    assert ei.value.code == nat.FPT_EUNSUPPORTED
    p = nat.make_params(model=nat.MODEL_POLYNOMIAL, precision="f32_kahan", poly=[-1.0, 0, 0.1], n_max=6.0)
    with pytest.raises(nat.FptError) as ei:  # V(phi_end = 1) < 0
        nat.fpt_simulate(p, 8, 4.0, 1.0, math.inf, 1e-3, 0.1, 0, x, x.clone())
    assert ei.value.code == nat.FPT_EINVAL
    with pytest.raises(ValueError):
        nat.make_params(model=nat.MODEL_POLYNOMIAL, poly=[0.0] * 9, n_max=6.0)


@pytest.mark.parametrize("precision", ["f64", "f32_kahan", "f32_f64acc"])
def test_polynomial_sets_in_one_batch(nat, precision):
    """Several sets of one potential (different phi_in, phi_end, walls and
    biases) in one batched launch give exactly the records of one call per
    set (the coefficients go into every set's constants)."""
    import torch
    from paper_2206_11234_gb300 import workloads as W
    c = [0, 0, 0.5 * 0.3, 0, 0.25 * 0.02]
    specs = [W.SetSpec(phi_in=3.5, phi_end=1.6, m=0.0, b=0.5, dN=1e-3, n_max=20.0, n_traj=1500, model=2, set_id=0),
             W.SetSpec(phi_in=3.0, phi_end=1.6, m=0.0, b=0.0, dN=1e-3, n_max=20.0, n_traj=999, phi_uv=3.2,
                       model=2, set_id=3),
             W.SetSpec(phi_in=4.0, phi_end=2.0, m=0.0, b=1.0, dN=2e-3, n_max=20.0, n_traj=1024, model=2, set_id=7)]
    p = nat.make_params(model=nat.MODEL_POLYNOMIAL, precision=precision, poly=c, n_max=20.0)
    n = sum(s.n_traj for s in specs)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty_like(N)
    nat.fpt_simulate_batch(p, nat.make_sets(specs), 4, N, lw)
    off = 0
    for s in specs:
        N1 = torch.empty(s.n_traj, dtype=torch.float64, device="cuda")
        l1 = torch.empty_like(N1)
        nat.fpt_simulate_batch(p, nat.make_sets([s]), 4, N1, l1)
        assert torch.equal(N[off:off + s.n_traj], N1), s.set_id
        assert torch.equal(lw[off:off + s.n_traj], l1), s.set_id
        off += s.n_traj
