"""Error paths exercised from the host, without faulting a GPU.

* An allocation the library makes fails as on a full device
  (fpt_inject_alloc_failures): the call returns FPT_ENOMEM and names the
  allocation, and the next call runs normally and reproduces a call made
  before the failure, for the batched stepper, the histogram, the host-buffer
  entry and the learned-bias training step.
* A status bit set in the device status word (fpt_inject_status, the path a
  device-side check or an expired tensor-core wait takes) makes the call
  return FPT_EDEVICE_STATUS with the bit in its message, and the next call
  succeeds.
"""
import numpy as np
import pytest

from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    yield native
    native.lib.fpt_inject_alloc_failures(0)
    native.lib.fpt_inject_status(0)


def _batch(nat, seed):
    import torch
    wl = W.drift_dominated_ladder(scale=1 / 4096)
    sets = nat.make_sets(wl.sets)
    n = wl.n_total
    nb = sum(s.n_bins for s in wl.sets)
    p = nat.make_params(precision="f32_kahan", m=0.01, n_max=10.0)
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty_like(N)
    bins = nat.empty_bins(nb)
    counts = nat.empty_counts(len(wl.sets))
    nat.fpt_simulate_batch(p, sets, seed, N, lw, bins, counts)
    return N.cpu().numpy(), lw.cpu().numpy(), bins.cpu().numpy(), counts.cpu().numpy()


def _same(ref, got):
    """Records and counters exactly; bin sums up to the order of their atomic additions."""
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and np.array_equal(ref[3], got[3])
    _same_bins(ref[2], got[2])


def _same_bins(a, b):
    assert np.array_equal(a[:, 0], b[:, 0]) and np.array_equal(a.view(np.int64)[:, 7], b.view(np.int64)[:, 7])
    np.testing.assert_allclose(b[:, 1:7], a[:, 1:7], rtol=1e-12, atol=1e-300)


def _expect(nat, code, fn, words):
    with pytest.raises(nat.FptError) as ei:
        fn()
    assert ei.value.code == code, ei.value
    msg = nat.lib.fpt_last_error().decode()
    for w in words:
        assert w in msg, msg


def test_allocation_failure_then_clean_call(nat):
    import torch
    ref = _batch(nat, 3)
    assert nat.lib.fpt_inject_alloc_failures(1) == nat.FPT_OK
    _expect(nat, nat.FPT_ENOMEM, lambda: _batch(nat, 3), ["workspace allocation"])
    _same(ref, _batch(nat, 3))
    # the histogram entry
    N = torch.from_numpy(ref[0]).cuda()
    lw = torch.from_numpy(ref[1]).cuda()
    bins, counts = nat.empty_bins(40), nat.empty_counts(1)
    nat.fpt_histogram(N, lw, 40, 7.0, 10.0, bins, counts)
    hb = bins.cpu().numpy()
    nat.lib.fpt_inject_alloc_failures(1)
    _expect(nat, nat.FPT_ENOMEM, lambda: nat.fpt_histogram(N, lw, 40, 7.0, 10.0, bins, counts),
            ["histogram workspace"])
    nat.fpt_histogram(N, lw, 40, 7.0, 10.0, bins, counts)
    _same_bins(hb, bins.cpu().numpy())
    # the host-buffer entry (its device buffers come from the library's pool)
    wl = W.drift_dominated_ladder(scale=1 / 4096)
    sets = nat.make_sets(wl.sets)
    p = nat.make_params(precision="f32_kahan", m=0.01, n_max=10.0)
    nb = sum(s.n_bins for s in wl.sets)
    hN = torch.empty(wl.n_total, dtype=torch.float64).pin_memory()
    hl = torch.empty_like(hN).pin_memory()
    hbins = torch.empty((nb, nat.BIN_FIELDS), dtype=torch.float64).pin_memory()
    hc = torch.empty((len(wl.sets), 4), dtype=torch.int64).pin_memory()
    nat.lib.fpt_inject_alloc_failures(1)
    _expect(nat, nat.FPT_ENOMEM, lambda: nat.fpt_simulate_batch_host(p, sets, 3, hN, hl, hbins, hc),
            ["device buffers"])
    nat.fpt_simulate_batch_host(p, sets, 3, hN, hl, hbins, hc)
    assert np.array_equal(hN.numpy(), ref[0]) and np.array_equal(hl.numpy(), ref[1])


def test_allocation_failure_in_training_step(nat):
    spec = W.SetSpec(phi_in=3.0, m=1.0, b=0.0, dN=1e-3, n_max=6.0, n_traj=2048, phi_uv=4.0)
    init = W.mlp_params(seed=31, gain=1.0, out_scale=0.05)
    init[-1] = 0.6
    norm = (3.5, 1.5, 2.5, 0.4)
    a = nat.MlpTrainer(spec, init, norm, k_eval=32)
    b = nat.MlpTrainer(spec, init, norm, k_eval=32)
    sa = a.step(seed=9, tail_N=2.0, lr=1e-3)
    nat.lib.fpt_inject_alloc_failures(1)
    with pytest.raises(nat.FptError) as ei:
        b.step(seed=9, tail_N=2.0, lr=1e-3)
    assert ei.value.code == nat.FPT_ENOMEM
    sb = b.step(seed=9, tail_N=2.0, lr=1e-3)
    # the failed step changed nothing: the retried step equals the first trainer's
    # (up to the order of the floating-point sums, which atomics leave open)
    assert sa["n_records"] == sb["n_records"]
    for k in ("log_second_moment", "p_hat", "frac_in_tail"):
        assert abs(sa[k] - sb[k]) <= 1e-9 * max(1.0, abs(sa[k])), k
    np.testing.assert_allclose(b.master.cpu().numpy(), a.master.cpu().numpy(), rtol=1e-5, atol=1e-7)


def test_injected_status_is_reported_then_clean_call(nat):
    ref = _batch(nat, 4)
    for bits in (0x1, 0x40):
        assert nat.lib.fpt_inject_status(bits) == nat.FPT_OK
        _expect(nat, nat.FPT_EDEVICE_STATUS, lambda: _batch(nat, 4), [f"0x{bits:x}"])
        _same(ref, _batch(nat, 4))
