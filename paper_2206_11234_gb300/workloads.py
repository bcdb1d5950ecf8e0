"""Seeded synthetic workloads and inputs (shared by the GPU path's tests and
the oracle's; holds none of the method's arithmetic).

The paper's runs are synthetic (no dataset): quadratic inflation
V = m^2 phi^2 / 2 with phi_end = sqrt(2) (§3), started at phi_in with an
optional reflecting wall phi_uv, biased with B = b S (§2.3).  The workloads
below have the shapes of the paper's three regimes (§3.1 diffusion
domination m >~ 1, §3.2 interim, §3.3 drift domination m << 1) at the sizes
this library is measured on.
"""
import dataclasses
import math
from typing import List, Optional

import numpy as np

PHI_END = math.sqrt(2.0)  # end of slow roll, epsilon_1 = 1 (§3)


@dataclasses.dataclass
class SetSpec:
    """One parameter set: n_traj runs sharing (model, phi_in, m, b, dN, ...)."""
    phi_in: float
    m: float
    b: float
    dN: float
    n_max: float
    n_traj: int
    phi_end: float = PHI_END
    phi_uv: float = math.inf
    set_id: int = 0
    hist_lo: float = 0.0
    hist_hi: float = 1.0
    n_bins: int = 100
    model: int = 0  # 0 quadratic, 1 constant drift/noise test model
    a0: float = 0.0
    s0: float = 0.0
    traj_offset: int = 0  # id of the set's first run (sharding across ranks)


@dataclasses.dataclass
class Workload:
    name: str
    sets: List[SetSpec]
    precision: str  # "f64", "f32_kahan", "f32_f64acc"
    seed: int = 0
    tail_N: Optional[float] = None  # tail event E = {N > tail_N} for effective sample size
    note: str = ""

    @property
    def n_total(self) -> int:
        return sum(s.n_traj for s in self.sets)


def quadratic_fixed_b(scale: float = 1.0) -> Workload:
    """m = 1, phi_in = 3, no wall, dN = 1e-3, b = 1, 16384 runs, FP64;
    100 bins on (0, 6]; runs still going at N = 6 are censored."""
    n = max(1, int(16384 * scale))
    s = SetSpec(phi_in=3.0, m=1.0, b=1.0, dN=1e-3, n_max=6.0, n_traj=n, hist_lo=0.0, hist_hi=6.0,
                n_bins=100)
    return Workload("quadratic m=1 phi_in=3 b=1 dN=1e-3, 16384 runs, FP64", [s], "f64", seed=0,
                    tail_N=3.0)


def drift_dominated_ladder(scale: float = 1.0, precision: str = "f32_kahan") -> Workload:
    """m = 0.01, phi_in = 6, dN = 1e-3, b in {0, 0.5, 1, 2, 4} x 2^22 runs in one
    launch; 400 bins on (7, 10]; censored at N = 10 (the histogram's upper edge)."""
    n = max(1, int((1 << 22) * scale))
    sets = [SetSpec(phi_in=6.0, m=0.01, b=b, dN=1e-3, n_max=10.0, n_traj=n, set_id=i, hist_lo=7.0,
                    hist_hi=10.0, n_bins=400) for i, b in enumerate((0.0, 0.5, 1.0, 2.0, 4.0))]
    # classical duration (phi_in^2 - phi_end^2)/4 = 8.5; sigma_N ~ 0.02 (§3.3 regime)
    return Workload(f"drift-dominated quadratic m=0.01 phi_in=6 dN=1e-3, b ladder 0/0.5/1/2/4 x {n}",
                    sets, precision, seed=0, tail_N=8.6)


def batched_uneven(scale: float = 1.0) -> Workload:
    """64 sets: phi_in = 2 * 10^(s/63), m = (0.01, 0.1, 1)[s % 3],
    b = (0, 1, 3)[(s // 3) % 3], 2^20 runs each, dN = 1e-3, FP32; 256 bins per
    set on (0, h_s] with h_s = 2 N_cl + 10, N_cl = (phi_in^2 - 2)/4, censored at h_s."""
    n = max(1, int((1 << 20) * scale))
    sets = []
    for s in range(64):
        phi_in = 2.0 * 10.0 ** (s / 63.0)
        n_cl = (phi_in**2 - 2.0) / 4.0
        hi = 2.0 * n_cl + 10.0
        sets.append(SetSpec(phi_in=phi_in, m=(0.01, 0.1, 1.0)[s % 3], b=(0.0, 1.0, 3.0)[(s // 3) % 3],
                            dN=1e-3, n_max=hi, n_traj=n, set_id=s, hist_lo=0.0, hist_hi=hi,
                            n_bins=256))
    return Workload(f"batched uneven: 64 sets x {n} runs, phi_in 2..20, m 0.01/0.1/1, b 0/1/3",
                    sets, "f32_kahan", seed=0)


def diffusion_wall(scale: float = 1.0, biases=(2.0, 4.0, 6.0)) -> Workload:
    """m = 1, phi_in = 8, reflecting wall phi_uv = 9, dN = 5e-4, 2^25 runs per
    bias; 512 bins on (0, 60]; censored at N = 60; FP32 state with FP64
    log-weight sums and crossing."""
    n = max(1, int((1 << 25) * scale))
    sets = [SetSpec(phi_in=8.0, m=1.0, b=b, dN=5e-4, n_max=60.0, n_traj=n, phi_uv=9.0, set_id=i,
                    hist_lo=0.0, hist_hi=60.0, n_bins=512) for i, b in enumerate(biases)]
    return Workload(f"diffusion-dominated quadratic m=1 phi_in=8 phi_uv=9 dN=5e-4, b {biases} x {n}",
                    sets, "f32_f64acc", seed=0, tail_N=40.0)


def constant_model(a0: float, s0: float, distance: float, b: float, dN: float, n_traj: int,
                   n_max: float) -> SetSpec:
    """Constant drift a0 < 0 and noise s0: the inverse-Gaussian test model."""
    return SetSpec(phi_in=1.0 + distance, phi_end=1.0, m=0.0, b=b, dN=dN, n_max=n_max,
                   n_traj=n_traj, model=1, a0=a0, s0=s0, hist_lo=0.0, hist_hi=n_max, n_bins=100)


def random_records(n: int, seed: int, lo: float, hi: float, censored_frac: float = 0.02,
                   logw_scale: float = 5.0):
    """Synthetic (N, log w) records for histogram tests: N spread over and
    around (lo, hi], some +inf (censored), log w roughly normal."""
    rng = np.random.default_rng(seed)
    span = hi - lo
    N = rng.uniform(lo - 0.1 * span, hi + 0.1 * span, size=n)
    N[rng.random(n) < censored_frac] = np.inf
    logw = rng.normal(-0.5 * logw_scale, logw_scale, size=n)
    return N, logw


def mlp_params(seed: int, hidden: int = 64, gain: float = 1.0, out_scale: float = 0.1):
    """Random MLP parameters in the packed order W1[h][2], b1[h], W2[h][h],
    b2[h], w3[h], b3 (float64; the caller rounds them to the storage type)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, gain / math.sqrt(2.0), size=(hidden, 2))
    b1 = rng.normal(0.0, 0.1, size=hidden)
    W2 = rng.normal(0.0, gain / math.sqrt(hidden), size=(hidden, hidden))
    b2 = rng.normal(0.0, 0.1, size=hidden)
    w3 = rng.normal(0.0, out_scale / math.sqrt(hidden), size=hidden)
    b3 = np.array([0.0])
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3])
