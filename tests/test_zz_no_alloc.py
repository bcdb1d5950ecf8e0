"""The no-allocation batched entry point (fpt_simulate_batch_noalloc) against
the regular one (fpt_simulate_batch).

It serves callers that must not allocate device memory while they run (all
device memory reserved by their own pool or budget, or latency-bound loops):
its scratch is a fixed array inside the library, shared by every call.  Two
calls in a row, with different sets and seeds, must each reproduce the
regular entry's records exactly (the same kernel runs on the same inputs, so
the tolerance the parity tests use for records of one launch shape, zero, is
the one applied here), which also shows that each call re-initialises the
shared scratch it inherits from the previous one.  This file is collected
last so that a failure here cannot hide another test's result.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    f = native.lib.fpt_simulate_batch_noalloc
    f.argtypes = [ctypes.POINTER(native.FptParams), ctypes.POINTER(native.FptSet), ctypes.c_int32,
                  ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return native


def _regular(nat, p, sets, seed, n):
    import torch
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    nat.fpt_simulate_batch(p, sets, seed, N, lw)
    return N.cpu().numpy(), lw.cpu().numpy()


def _noalloc(nat, p, sets, seed, n):
    import torch
    N = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    lw = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    rc = nat.lib.fpt_simulate_batch_noalloc(ctypes.byref(p), sets, len(sets), seed,
                                            ctypes.c_void_p(N.data_ptr()), ctypes.c_void_p(lw.data_ptr()))
    assert rc == nat.FPT_OK, nat.lib.fpt_last_error()
    return N.cpu().numpy(), lw.cpu().numpy()


def test_noalloc_matches_regular_entry_twice_in_a_row(nat):
    import torch
    # call 1: drift-dominated ladder (5 sets); call 2: wall + several masses (12 sets)
    wl1 = W.drift_dominated_ladder(scale=1 / 2048)
    wl2 = W.batched_uneven(scale=1 / 2048)
    specs2 = wl2.sets[::5]
    specs2[0].phi_uv = specs2[0].phi_in * 1.1
    for specs, seed, prec in ((wl1.sets, 11, "f32_kahan"), (specs2, 12, "f32_f64acc"),
                              (wl1.sets[:2], 13, "f64")):
        sets = nat.make_sets(specs)
        n = sum(s.n_traj for s in specs)
        steps_a = torch.zeros(1, dtype=torch.int64, device="cuda")
        steps_b = torch.zeros(1, dtype=torch.int64, device="cuda")
        pa = nat.make_params(precision=prec, m=specs[0].m, n_max=specs[0].n_max, steps_out=steps_a)
        pb = nat.make_params(precision=prec, m=specs[0].m, n_max=specs[0].n_max, steps_out=steps_b)
        Nr, lwr = _regular(nat, pa, sets, seed, n)
        Nn, lwn = _noalloc(nat, pb, sets, seed, n)
        np.testing.assert_array_equal(Nn, Nr)
        np.testing.assert_array_equal(lwn, lwr)
        assert steps_a.item() == steps_b.item() > 0


def test_noalloc_rejects_more_sets_than_its_scratch_holds(nat):
    import torch
    specs = W.batched_uneven(scale=1 / 4096).sets  # 64 sets > the fixed capacity
    sets = nat.make_sets(specs)
    p = nat.make_params(precision="f32_kahan", m=1.0, n_max=10.0)
    x = torch.empty(sum(s.n_traj for s in specs), dtype=torch.float64, device="cuda")
    rc = nat.lib.fpt_simulate_batch_noalloc(ctypes.byref(p), sets, len(sets), 0,
                                            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()))
    assert rc == nat.FPT_EINVAL
    assert b"at most" in nat.lib.fpt_last_error()


def test_noalloc_power_bias_and_no_step_counter(nat):
    """The power-law bias (its own stepper instantiation and set-table fields)
    and a call without the optional step counter (steps_out = NULL) also
    reproduce the regular entry bit for bit."""
    specs = [W.SetSpec(phi_in=6.0, m=1e-3, b=0.0, dN=1e-4, n_max=40.0, n_traj=3000, set_id=0),
             W.SetSpec(phi_in=5.5, m=1e-3, b=0.0, dN=1e-4, n_max=40.0, n_traj=1500, set_id=1)]
    specs[0].b = 2.0e-6
    specs[1].b = 1.0e-6
    sets = nat.make_sets(specs)
    n = sum(s.n_traj for s in specs)
    for prec, bias_p in (("f32_f64acc", 3.0), ("f64", 2.5)):
        p = nat.make_params(precision=prec, m=1e-3, n_max=40.0, bias_p=bias_p)
        Nr, lwr = _regular(nat, p, sets, 21, n)
        Nn, lwn = _noalloc(nat, p, sets, 21, n)
        assert np.isfinite(Nr).mean() > 0.5
        np.testing.assert_array_equal(Nn, Nr)
        np.testing.assert_array_equal(lwn, lwr)
    p = nat.make_params(precision="f32_kahan", m=0.01, n_max=10.0)  # steps_out NULL
    wl = W.drift_dominated_ladder(scale=1 / 4096)
    sets = nat.make_sets(wl.sets)
    n = wl.n_total
    Nr, lwr = _regular(nat, p, sets, 22, n)
    Nn, lwn = _noalloc(nat, p, sets, 22, n)
    np.testing.assert_array_equal(Nn, Nr)
    np.testing.assert_array_equal(lwn, lwr)
