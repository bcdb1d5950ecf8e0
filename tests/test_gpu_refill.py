"""The persistent scheduler under load: many more runs than resident lanes, so
lanes refill from the ticket counter many times and finished runs are
replayed while their warp-mates are still running (their state parked in
shared memory).  Per-run parity with the oracle on ids spread over the whole
range, and binary32 against binary64 on every run."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _gpu(nat, n, precision, **kw):
    import torch
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = nat.make_params(precision=precision, m=kw["m"], n_max=kw["n_max"], steps_out=steps,
                        k_steps=kw.get("k_steps", 0), block_dim=kw.get("block_dim", 0))
    nat.fpt_simulate(p, n, kw["phi_in"], SQ2, kw.get("phi_uv", math.inf), kw["dN"], kw["b"], kw.get("seed", 0),
                     N, lw)
    return N.cpu().numpy(), lw.cpu().numpy(), int(steps.item())


@pytest.mark.parametrize("case", [
    dict(phi_in=1.6, m=1.0, b=0.5, dN=1e-3, n_max=5.0),               # short runs (~150 steps)
    dict(phi_in=3.0, m=1.0, b=1.0, dN=1e-3, n_max=6.0, phi_uv=3.4),   # long, with a wall
], ids=["short", "long_wall"])
def test_refills_f64_per_run_parity_on_spread_ids(nat, case):
    n = 1 << 20 if case["phi_in"] < 2 else 1 << 19
    N, lw, _ = _gpu(nat, n, "f64", **case)
    ids = np.unique(np.linspace(0, n - 1, 1500).astype(np.int64))
    bad = 0
    for i in ids:
        r = oracle.make_run(m=case["m"], phi_in=case["phi_in"], phi_uv=case.get("phi_uv", math.inf),
                            dN=case["dN"], b=case["b"], n_max=case["n_max"], traj_offset=int(i))
        No, lo, so = oracle.simulate(r, 1)
        if np.isinf(No[0]) != np.isinf(N[i]):
            bad += 1
            continue
        scale = max(1.0, 0.5 * so[0] * (case["b"] * math.sqrt(case["dN"]) * 0.8 + 0.5 * case["b"] ** 2 * case["dN"]))
        if (np.isfinite(No[0]) and abs(N[i] - No[0]) > 1e-12 * No[0]) or abs(lw[i] - lo[0]) > 1e-12 * scale:
            bad += 1
    assert bad == 0, f"{bad} of {ids.size} runs differ"


@pytest.mark.parametrize("precision", ["f32_kahan", "f32_f64acc"])
def test_refills_f32_tracks_f64_on_every_run(nat, precision):
    case = dict(phi_in=1.6, m=1.0, b=0.5, dN=1e-3, n_max=5.0)
    n = 1 << 20
    N64, lw64, s64 = _gpu(nat, n, "f64", **case)
    N32, lw32, s32 = _gpu(nat, n, precision, **case)
    fin = np.isfinite(N64) & np.isfinite(N32)
    assert fin.mean() > 0.999
    dN = np.abs(N32[fin] - N64[fin])
    assert np.mean(dN < case["dN"]) > 0.995  # same crossing step (a few flips allowed)
    dl = np.abs(lw32 - lw64)
    # a corrupted running sum would shift ln w by O(1) on many runs; a crossing
    # flip moves it by one step's b sqrt(dN) xi (< 0.2)
    assert np.quantile(dl, 0.99) < 0.05
    assert np.max(dl) < 0.2
    assert np.median(dl) < 1e-5
    assert abs(s32 / s64 - 1) < 1e-3
