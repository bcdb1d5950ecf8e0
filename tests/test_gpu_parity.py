"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

* Philox words: bit-exact.  Normals: binary64 within a few ulp (CUDA's and
  glibc's log/sin/cos differ by an ulp or two); binary32 (hardware
  approximations, 23-bit uniform) within ~1e-6 in the bulk.
* FP64 stepper, per run: same crossing step for every run (n * 1e-6 < 1 at
  these sizes), |dN| <= 1e-12 N and |d ln w| <= 1e-12 max(1, sum_m |increment_m|).
* Reduced precision: statistical parity (every histogram bin within 3 combined
  sigma, <N> to 1e-3 relative) plus a per-run error report against FP64.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_11234_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)


@pytest.fixture(scope="module")
def nat(cuda_device):
    from paper_2206_11234_gb300 import native
    return native


def gpu_run(nat, *, n, phi_in, dN, b, n_max, m=1.0, phi_uv=math.inf, phi_end=SQ2, seed=0,
            precision="f64", model=0, a0=0.0, s0=0.0, set_id=0, traj_offset=0, block_dim=0,
            k_steps=0):
    import torch
    N = torch.empty(n, dtype=torch.float64, device="cuda")
    lw = torch.empty(n, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = nat.make_params(model=model, precision=precision, m=m, a0=a0, s0=s0, n_max=n_max,
                        set_id=set_id, traj_offset=traj_offset, block_dim=block_dim, k_steps=k_steps,
                        steps_out=steps)
    nat.fpt_simulate(p, n, phi_in, phi_end, phi_uv, dN, b, seed, N, lw)
    torch.cuda.synchronize()
    return N.cpu().numpy(), lw.cpu().numpy(), int(steps.item())


def oracle_run(*, n, phi_in, dN, b, n_max, m=1.0, phi_uv=math.inf, phi_end=SQ2, seed=0, model=0,
               a0=0.0, s0=0.0, set_id=0, traj_offset=0, **_):
    r = oracle.make_run(model=model, m=m, a0=a0, s0=s0, phi_in=phi_in, phi_end=phi_end,
                        phi_uv=phi_uv, dN=dN, b=b, n_max=n_max, seed=seed, set_id=set_id,
                        traj_offset=traj_offset)
    return oracle.simulate(r, n)


def assert_f64_parity(N_g, lw_g, N_o, lw_o, steps_o, b, dN):
    same_inf = np.isinf(N_g) == np.isinf(N_o)
    assert same_inf.all(), f"{(~same_inf).sum()} runs differ in censoring"
    fin = np.isfinite(N_o)
    dn = np.abs(N_g[fin] - N_o[fin])
    bad_N = dn > 1e-12 * np.maximum(N_o[fin], 1e-300)
    bad_N |= (N_o[fin] == 0) & (N_g[fin] != 0)
    # sum over steps of |b sqrt(dN) xi| + b^2 dN/2, with E|xi| = sqrt(2/pi), halved for safety
    scale = np.maximum(1.0, 0.5 * steps_o * (abs(b) * math.sqrt(dN) * math.sqrt(2 / math.pi)
                                             + 0.5 * b * b * dN))
    bad_lw = np.abs(lw_g - lw_o) > 1e-12 * scale
    n_bad = int(bad_N.sum() + bad_lw.sum())
    assert n_bad <= 1e-6 * N_o.size, (
        f"{bad_N.sum()} N and {bad_lw.sum()} log w mismatches; max dN {dn.max() if dn.size else 0}")


def test_philox_words_bit_exact(nat):
    import torch
    out = torch.empty(4 * 4096, dtype=torch.int32, device="cuda")
    for seed, traj, set_id in ((0, 0, 0), (0x123456789ABCDEF, 2**40 + 77, 5), (2**64 - 1, 2**64 - 1, 2**32 - 1)):
        nat.fpt_normals(seed, traj, set_id, 1000, 4096, 3, out)
        got = out.cpu().numpy().view(np.uint32).reshape(-1, 4)
        for k in (0, 1, 17, 4095):
            ref = oracle.philox4x32_10([1000 + k, traj & 0xFFFFFFFF, traj >> 32, set_id],
                                       [seed & 0xFFFFFFFF, seed >> 32])
            assert np.array_equal(got[k], ref), (seed, traj, k)


def test_normals_match_oracle(nat):
    import torch
    nb = 2048
    o64 = torch.empty(4 * nb, dtype=torch.float64, device="cuda")
    o32 = torch.empty(4 * nb, dtype=torch.float32, device="cuda")
    nat.fpt_normals(7, 12345, 3, 0, nb, "f64", o64)
    nat.fpt_normals(7, 12345, 3, 0, nb, "f32_kahan", o32)
    ref = np.concatenate([oracle.normals4(7, 12345, 3, k) for k in range(nb)])
    g64 = o64.cpu().numpy()
    g32 = o32.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g64 - ref) / np.maximum(np.abs(ref), 1e-3)) < 4e-15
    # binary32 error budget per normal, from the pair radius r = sqrt(xi0^2 + xi1^2):
    # the 23-bit uniform moves -2 ln u0 by <= 2^-23 e^{r^2/2}, lg2.approx by <= 2^-22 ln 4,
    # both divided by 2r in r; the angle (quantised u1, binary32 2 pi, sin/cos.approx)
    # is good to ~1.5e-6 rad
    r = np.repeat(np.hypot(ref[0::2], ref[1::2]), 2)
    bound = (2.0**-23 * np.exp(r * r / 2) + 2.0**-22 * 1.3863) / (2 * r) + 1.5e-6 * r + 1e-6
    err = np.abs(g32 - ref)
    assert np.all(err < 2 * bound), np.max(err / bound)
    assert np.median(err) < 1e-6
    assert np.all(np.abs(g32) < 5.78)  # largest binary32 radius: sqrt(2 ln 2^24)


CASES_F64 = [
    # config-1 shape: m = 1, phi_in = 3, b = 1, no wall, dN = 1e-3, censored at 6
    dict(n=16384, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0),
    dict(n=3001, phi_in=3.0, dN=1e-3, b=0.0, n_max=6.0),
    dict(n=2000, phi_in=3.0, dN=1e-3, b=0.8, n_max=40.0, phi_uv=3.3),
    dict(n=1000, phi_in=3.0, dN=1e-3, b=1.0, n_max=0.5),  # mostly censored
    dict(n=1537, model=1, a0=-1.0, s0=0.5, phi_in=2.0, phi_end=1.0, dN=1e-3, b=0.7, n_max=20.0),
    dict(n=777, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0, seed=12345, set_id=9, traj_offset=2**33 + 5),
]


@pytest.mark.parametrize("case", CASES_F64, ids=lambda c: f"n{c['n']}_b{c['b']}")
def test_f64_per_run_parity(nat, case):
    N_g, lw_g, steps_g = gpu_run(nat, precision="f64", **case)
    N_o, lw_o, steps_o = oracle_run(**case)
    assert steps_g == int(steps_o.sum())
    assert_f64_parity(N_g, lw_g, N_o, lw_o, steps_o, case["b"], case["dN"])


@pytest.mark.parametrize("precision,block_dim,k_steps", [("f64", 32, 4), ("f64", 512, 4),
                                                         ("f64", 64, 8), ("f32_kahan", 64, 64),
                                                         ("f32_f64acc", 512, 32)])
def test_results_independent_of_launch_shape(nat, precision, block_dim, k_steps):
    """Records do not depend on the block size; the block length k_steps only
    changes how the normals' running sum is associated (last bits of ln w in
    binary64; binary32 block sums are rounded per block)."""
    case = dict(n=2049, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0)
    N_g, lw_g, _ = gpu_run(nat, precision=precision, block_dim=block_dim, k_steps=k_steps, **case)
    ks_default = 4 if precision == "f64" else 16
    N_ref, lw_ref, _ = gpu_run(nat, precision=precision, k_steps=k_steps, **case)
    assert np.array_equal(N_g, N_ref) and np.array_equal(lw_g, lw_ref)
    N_d, lw_d, _ = gpu_run(nat, precision=precision, k_steps=ks_default, **case)
    assert np.array_equal(N_g, N_d)
    tol = 1e-12 if precision == "f64" else 1e-4
    assert np.max(np.abs(lw_g - lw_d)) < tol * max(1.0, np.abs(lw_d).max())


def test_degenerate_inputs(nat):
    # start at (or below) the end of inflation
    for phi_in in (SQ2, 1.0):
        N, lw, st = gpu_run(nat, n=100, phi_in=phi_in, dN=1e-3, b=1.0, n_max=6.0)
        assert np.all(N == 0) and np.all(lw == 0) and st == 0
    # one run; every binary32 block length
    for prec in ("f64", "f32_kahan", "f32_f64acc"):
        N, lw, st = gpu_run(nat, n=1, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0, precision=prec)
        assert np.isfinite(N[0]) and st > 0
    # b = 0: log w exactly 0 in every precision
    for prec in ("f64", "f32_kahan", "f32_f64acc"):
        N, lw, _ = gpu_run(nat, n=500, phi_in=3.0, dN=1e-3, b=0.0, n_max=6.0, precision=prec)
        assert np.all(lw == 0.0)
    # a cap of one step: everything censored after exactly one step
    N, lw, st = gpu_run(nat, n=64, phi_in=3.0, dN=1e-3, b=1.0, n_max=1e-3)
    assert np.all(np.isinf(N)) and st == 64


def test_sharding_by_trajectory_offset_is_exact(nat):
    a = gpu_run(nat, n=5000, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0, precision="f32_kahan")
    b = gpu_run(nat, n=3000, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0, precision="f32_kahan",
                traj_offset=2000)
    assert np.array_equal(a[0][2000:], b[0]) and np.array_equal(a[1][2000:], b[1])


def _pdf_and_sigma(bins, counts_total, lo, hi):
    nb = bins.shape[0]
    width = (hi - lo) / nb
    mx = bins[:, 0]
    with np.errstate(over="ignore", invalid="ignore"):
        s1 = np.where(np.isfinite(mx), np.exp(mx) * bins[:, 1], 0.0)
        s2 = np.where(np.isfinite(mx), np.exp(2 * mx) * bins[:, 2], 0.0)
    n = counts_total
    P = s1 / (width * n)
    var = np.maximum(s2 / n - (s1 / n) ** 2, 0.0) / n
    return P, np.sqrt(var) / width


@pytest.mark.parametrize("precision", ["f32_kahan", "f32_f64acc"])
def test_f32_statistical_parity_with_oracle(nat, precision):
    """Reduced precision against the FP64 oracle on the same seeds: per-run
    errors are reported (and bounded), every bin is within 3 combined sigma and
    <N> agrees to 1e-3."""
    case = dict(n=16384, phi_in=3.0, dN=1e-3, b=1.0, n_max=6.0)
    N_g, lw_g, _ = gpu_run(nat, precision=precision, **case)
    N_o, lw_o, st_o = oracle_run(**case)
    fin = np.isfinite(N_o) & np.isfinite(N_g)
    same_step = np.abs(N_g[fin] - N_o[fin]) < case["dN"]
    assert same_step.mean() > 0.99
    assert np.median(np.abs(N_g[fin] - N_o[fin])) < 1e-4
    assert np.median(np.abs(lw_g - lw_o)) < 1e-3
    assert abs(N_g[fin].mean() / N_o[fin].mean() - 1) < 1e-3
    bg, cg = oracle.histogram(N_g, lw_g, 100, 0.0, 6.0)
    bo, co = oracle.histogram(N_o, lw_o, 100, 0.0, 6.0)
    Pg, sg = _pdf_and_sigma(bg[0], case["n"], 0.0, 6.0)
    Po, so = _pdf_and_sigma(bo[0], case["n"], 0.0, 6.0)
    sig = np.hypot(sg, so)
    ok = (np.abs(Pg - Po) <= 3 * sig) | (sig == 0) & (Pg == Po)
    assert ok.all(), np.nonzero(~ok)


@pytest.mark.parametrize("precision", ["f32_kahan", "f32_f64acc"])
def test_f32_drift_dominated_matches_f64_gpu(nat, precision):
    """Drift-dominated ladder (m = 0.01, phi_in = 6): binary32 state against the
    binary64 GPU path on the same runs; b = 4 is ~10 sigma into the tail."""
    import torch
    for b in (0.0, 4.0):
        case = dict(n=4096, phi_in=6.0, dN=1e-3, b=b, n_max=10.0, m=0.01)
        N32, lw32, _ = gpu_run(nat, precision=precision, **case)
        N64, lw64, _ = gpu_run(nat, precision="f64", **case)
        assert np.all(np.isfinite(N32)) and np.all(np.isfinite(N64))
        assert abs(N32.mean() / N64.mean() - 1) < 1e-4
        assert np.max(np.abs(N32 - N64)) < 0.02 * 0.0203  # a few percent of sigma_N
        # per-run log-weight error: tiny unless the binary32 run crosses one step
        # earlier or later (then ln w moves by one step's increment)
        # (binary32 phi drifts ~2e-5 from binary64 over ~8600 steps, against a last
        # step of ~1.4e-3, so a few percent of runs flip)
        dl = np.abs(lw32 - lw64)
        flip = dl > 1e-3 * max(1.0, b)
        assert np.median(dl) < 1e-4 * max(1.0, b)
        assert np.mean(flip) < 0.05
        assert np.max(dl) < 1.5 * b * math.sqrt(1e-3) * 6 + 1e-3
        # statistically the two precisions agree bin by bin (400 bins on (7, 10])
        b32, _ = oracle.histogram(N32, lw32, 400, 7.0, 10.0)
        b64, _ = oracle.histogram(N64, lw64, 400, 7.0, 10.0)
        P32, s32 = _pdf_and_sigma(b32[0], N32.size, 7.0, 10.0)
        P64, s64 = _pdf_and_sigma(b64[0], N64.size, 7.0, 10.0)
        sig = np.hypot(s32, s64)
        assert np.all((np.abs(P32 - P64) <= 3 * sig) | ((sig == 0) & (P32 == P64)))
