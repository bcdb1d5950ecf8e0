"""The bounded waits of the tensor-core kernels, made to run out on purpose:
the library's own wait on an mbarrier that nothing arrives at gives up after
2^18 attempts (about a second), reports the expiry and returns; the context
stays usable (a learned-bias call succeeds after it)."""
import math

import pytest

from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def test_wait_expires_and_reports(nat):
    import torch
    expired, seconds = nat.fpt_wait_selftest()
    print(f"bounded wait expired={expired} after {seconds:.2f} s")
    assert expired
    assert 0.05 < seconds < 5.0
    # the context is still usable: a small learned-bias run goes through
    w = nat.mlp_pack(W.mlp_params(seed=1), (3.0, 1.0, 2.0, 0.5))
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=4096, phi_uv=4.0)
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=6.0, mlp=w, k_eval=32)
    N = torch.empty(4096, dtype=torch.float64, device="cuda")
    lw = torch.empty_like(N)
    nat.fpt_simulate_mlp(p, nat.make_sets([spec]), 0, N, lw)
    assert torch.isfinite(N).float().mean().item() > 0.99 and math.isfinite(lw.sum().item())
