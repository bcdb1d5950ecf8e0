"""Learned-bias MLP kernels (tcgen05 tensor cores) against the FP64 oracle MLP
evaluated with the same BF16-rounded parameters.

Tolerances come from the BF16 activations fed to the tensor cores (relative
rounding 2^-9 of h1 and delta2) and tanh.approx (~2^-11): per output
|db| ~ sqrt(64) |W2| |h1| 2^-10 |w3| sqrt(64) ~ 1e-3 sum|w3| / 8.  A wrong
operand layout, descriptor or transposition gives errors of the size of b itself.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NORM = (5.0, 0.35, 30.0, 1.0 / 30.0)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(1.4, 9.0, n).astype(np.float32)
    N = rng.uniform(0.0, 60.0, n).astype(np.float32)
    g = rng.normal(0.0, 1.0, n).astype(np.float32)
    return phi, N, g


@pytest.mark.parametrize("n", [1, 127, 129, 1000, 20000])
def test_mlp_forward_matches_oracle(nat, n):
    import torch
    params = W.mlp_params(seed=11, gain=1.5, out_scale=1.0)
    w = nat.mlp_pack(params, NORM)
    p64 = nat.mlp_unpack_bf16(params).numpy()
    phi, N, _ = _inputs(n, seed=n)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    nat.fpt_mlp_forward(w, torch.from_numpy(phi).cuda(), torch.from_numpy(N).cuda(), out)
    got = out.cpu().numpy().astype(np.float64)
    m = n
    ref = np.array([oracle.mlp_forward(p64, NORM, float(phi[i]), float(N[i]))[0] for i in range(m)])
    scale = np.abs(p64[-65:-1]).sum()
    err = np.abs(got[:m] - ref)
    assert err.max() < 4e-3 * scale, (err.max(), scale)
    assert err.mean() < 1e-3 * scale
    if m >= 100:  # the outputs vary far more than the error: the comparison has teeth
        assert np.std(ref) > 20 * err.mean()


@pytest.mark.parametrize("n", [1, 130, 2000])
def test_mlp_backward_matches_oracle(nat, n):
    import torch
    params = W.mlp_params(seed=12, gain=1.5, out_scale=1.0)
    w = nat.mlp_pack(params, NORM)
    p64 = nat.mlp_unpack_bf16(params).numpy()
    phi, N, g = _inputs(n, seed=100 + n)
    grad = torch.zeros(nat.MLP_NPARAM, dtype=torch.float32, device="cuda")
    nat.fpt_mlp_backward(w, torch.from_numpy(phi).cuda(), torch.from_numpy(N).cuda(),
                         torch.from_numpy(g).cuda(), grad)
    got = grad.cpu().numpy().astype(np.float64)
    ref = np.zeros(nat.MLP_NPARAM)
    for i in range(n):
        ref += oracle.mlp_backward(p64, NORM, float(phi[i]), float(N[i]), float(g[i]))
    H = 64
    groups = {"W1": slice(0, 2 * H), "b1": slice(2 * H, 3 * H), "W2": slice(3 * H, 3 * H + H * H),
              "b2": slice(3 * H + H * H, 4 * H + H * H), "w3": slice(4 * H + H * H, 5 * H + H * H),
              "b3": slice(5 * H + H * H, 5 * H + H * H + 1)}
    for name, sl in groups.items():
        r, q = ref[sl], got[sl]
        nr = np.linalg.norm(r)
        assert np.linalg.norm(q - r) <= 0.02 * nr + 1e-6, (name, np.linalg.norm(q - r), nr)
        assert np.max(np.abs(q - r)) <= 0.05 * np.max(np.abs(r)) + 1e-6, name
    # accumulation: a second call adds the same gradient again
    nat.fpt_mlp_backward(w, torch.from_numpy(phi).cuda(), torch.from_numpy(N).cuda(),
                         torch.from_numpy(g).cuda(), grad)
    got2 = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got2 - 2 * got) <= 1e-4 * np.linalg.norm(got) + 1e-6


def test_mlp_rejects_bad_arguments(nat):
    import torch
    params = W.mlp_params(seed=1)
    w = nat.mlp_pack(params, NORM)
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    assert nat.lib.fpt_mlp_forward(None, x.data_ptr(), x.data_ptr(), 4, x.data_ptr(), None) == nat.FPT_EINVAL
    assert nat.lib.fpt_mlp_forward(w.data_ptr() + 4, x.data_ptr(), x.data_ptr(), 4, x.data_ptr(),
                                   None) == nat.FPT_EINVAL  # misaligned parameters
    assert nat.lib.fpt_mlp_backward(w.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), -1, x.data_ptr(),
                                    None) == nat.FPT_EINVAL
    nat.fpt_mlp_forward(w, x[:0], x[:0], x[:0])  # n = 0 is a no-op
