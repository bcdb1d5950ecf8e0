"""The launch-shape autotuner: picks a shape from its candidate set, caches it
for calls that leave the shape at 0, and never changes the records."""
import numpy as np
import pytest

from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    yield native
    native.fpt_autotune_reset()


def test_autotune_picks_a_candidate_and_is_used(nat):
    import torch
    wl = W.drift_dominated_ladder(scale=1 / 256)
    sets = nat.make_sets(wl.sets)
    p = nat.make_params(precision="f32_kahan", m=0.01, n_max=10.0)
    nat.fpt_autotune_reset()
    N0, lw0, _, _ = nat.simulate_workload(wl, with_hist=False)  # defaults
    b, k, rate = nat.fpt_autotune(p, sets, seed=5, fraction=0.05)
    assert b in (128, 256, 512) and k in (8, 16, 32, 64) and rate > 1e9
    N1, lw1, _, _ = nat.simulate_workload(wl, with_hist=False)  # tuned shape
    N2, lw2, _, _ = nat.simulate_workload(wl, with_hist=False, block_dim=b, k_steps=k)
    assert torch.equal(N1, N2) and torch.equal(lw1, lw2)
    assert torch.equal(N0, N1)  # first-passage times never depend on the shape
    assert torch.max(torch.abs(lw0 - lw1)).item() < 1e-4 * max(1.0, torch.max(torch.abs(lw0)).item())


def test_autotune_f64_and_rejects_bad_fraction(nat):
    wl = W.quadratic_fixed_b(scale=0.25)
    sets = nat.make_sets(wl.sets)
    p = nat.make_params(precision="f64", m=1.0, n_max=6.0)
    b, k, rate = nat.fpt_autotune(p, sets, fraction=0.5)
    assert b in (128, 256, 512) and k in (4, 8) and rate > 0
    for f in (0.0, 1.5):
        with pytest.raises(nat.FptError):
            nat.fpt_autotune(p, sets, fraction=f)
