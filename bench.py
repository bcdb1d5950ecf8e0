"""Throughput of the importance-sampled first-passage-time hot path on GB300.

One step = one batched call of the C ABI over the whole workload: the
persistent Euler–Maruyama stepper for every run of every parameter set plus
the per-set weighted histograms.  Default workload: the drift-dominated bias
ladder, quadratic inflation m = 0.01, phi_in = 6, dN = 1e-3,
b in {0, 0.5, 1, 2, 4} x 2^22 runs in one launch, binary32 state with a
compensated log-weight sum, 400 bins on (7, 10].

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("trajectory steps/s and far-tail effective samples/s at 1 GB300 vs FP64 plain; "
          "% issue roofline")

# Algorithmic work per Euler–Maruyama step of the binary32 stepper (hand
# count of what one step needs, in warp-instructions per warp-step of 32 runs):
# Philox 38 per counter (10 rounds of two wide multiplies and the key/word
# mixing, less the per-run part of round 1), three counters per 16 steps;
# Box–Muller 16 per pair of steps (uniform and radius 4, angle word and angle
# 6 with the sine and cosine, the noise factor, the noise sum 2, ...); and 5.5
# for the update in psi = phi / sqrt(2 dN) (reciprocal, one FMA, one add), the
# noise term t, half a three-way block minimum and the noise sum.
ALG_INST_PER_STEP = 3 * 38 / 16 + 16 / 2 + 5.5
MUFU_PER_STEP = 3.0  # lg2 + sqrt + sin + cos per 2 steps, rcp per step
WIDE_MUL_PER_STEP = 3 * 19 / 16  # 32x32->64 multiplies: 19 per Philox counter (round 1 folds one)
ISSUE_PER_SM_CLK = 4.0  # warp-instructions issued per SM per clock (4 schedulers)
# learned bias: per run and evaluation, 2 x 64 tanh on the XU pipe and
# 2*64 + 64*64 + 64 multiply-adds (2 -> 64 -> 64 -> 1) on the tensor cores
MLP_TANH_PER_EVAL = 128
MLP_MAC_PER_EVAL = 2 * 64 + 64 * 64 + 64


# Sources the binary32 stepper kernel is built from: DRAM counters recorded
# for it in profiles/ apply only while their code is unchanged (the C++
# sources are compared without comments and blank lines; build.py, which
# holds the compiler flags, as it is).
STEPPER_SOURCES = ("stepper.cuh", "stepper_f32.cu", "stepper_f64.cu", "stepper_types.h", "rng.cuh", "stepper_launch.h",
                   "../build.py")


def strip_c_comments(text: str) -> str:
    """C/C++ source without // and /* */ comments, trailing blanks and blank
    lines (string and character literals are kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (ln.rstrip() for ln in "".join(out).split("\n"))
    return "\n".join(ln for ln in lines if ln)


def stepper_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2206_11234_gb300", "csrc")
    for f in STEPPER_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            text = fh.read()
        if not f.endswith(".py"):
            text = strip_c_comments(text)
        h.update(f.encode() + b"\0" + text.encode())
    return h.hexdigest()


def stepper_counters(precision, block_dim, k_steps, name="stepper_counters.json"):
    """The ncu counters recorded for a stepper kernel in profiles/ (DRAM bytes,
    instructions, pipe activity, branch and lane efficiency of one launch over
    a stated number of runs and steps), or None when no record matches this
    kernel's precision, launch shape (threads per block and block length) and
    source."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", name)
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if (rec.get("precision"), rec.get("block_dim"), rec.get("k_steps")) != (precision, block_dim, k_steps):
        return None
    if rec.get("source_sha256") != stepper_source_hash():
        return None
    return rec


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="drift_ladder",
                    choices=["drift_ladder", "quadratic_b1", "batched_uneven", "diffusion_wall",
                             "learned_bias", "estimators", "power_bias", "multi_bias"])
    ap.add_argument("--train-steps", type=int, default=4096, help="learned_bias: Adam steps")
    ap.add_argument("--train-runs", type=int, default=1 << 14, help="learned_bias: runs per Adam step")
    ap.add_argument("--lr", type=float, default=3e-3, help="learned_bias: Adam learning rate")
    ap.add_argument("--k-eval", type=int, default=64, choices=(16, 32, 64, 128),
                    help="learned_bias: steps between two evaluations of the bias network")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's runs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="default workload: skip the learned-bias experiment")
    ap.add_argument("--block-dim", type=int, default=0)
    ap.add_argument("--k-steps", type=int, default=0)
    return ap.parse_args()


def make_workload(name, scale):
    from paper_2206_11234_gb300 import workloads as W
    return {"drift_ladder": W.drift_dominated_ladder, "quadratic_b1": W.quadratic_fixed_b,
            "batched_uneven": W.batched_uneven, "diffusion_wall": W.diffusion_wall}[name](scale)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)
        return False

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons, "samples": len(self.rows)}


def tail_neff(N, lw, specs, tail_N):
    """n_eff = P^2 / Var(P) of the weighted estimator of P(N > tail_N), per set."""
    import torch
    out = []
    off = 0
    for s in specs:
        n = s.n_traj
        x = torch.where(N[off:off + n] > tail_N, torch.exp(lw[off:off + n]), torch.zeros_like(lw[off:off + n]))
        P = x.mean().item()
        var = x.var().item() / n if n > 1 else float("inf")
        out.append({"b": s.b, "P": P, "n_eff": (P * P / var) if var > 0 else 0.0})
        off += n
    return out


def cpu_oracle_rate(workload, seconds, threads=None):
    """The FP64 oracle on the host cores (threads calling the C oracle on
    disjoint run ranges; ctypes releases the GIL).  Returns (steps/s, cores,
    sample description)."""
    import numpy as np
    import oracle
    threads = threads or os.cpu_count() or 1
    specs = workload.sets
    lock = threading.Lock()
    tally = {"steps": 0, "runs": 0}
    deadline = time.perf_counter() + seconds
    next_index = [0] * len(specs)

    def worker(tid):
        chunk = 64
        j = tid % len(specs)
        while time.perf_counter() < deadline:
            s = specs[j]
            with lock:
                start = next_index[j]
                next_index[j] += chunk
            r = oracle.make_run(model=s.model, m=s.m, a0=s.a0, s0=s.s0, phi_in=s.phi_in,
                                phi_end=s.phi_end, phi_uv=s.phi_uv, dN=s.dN, b=s.b, n_max=s.n_max,
                                seed=workload.seed, set_id=s.set_id, traj_offset=start)
            _, _, st = oracle.simulate(r, chunk)
            with lock:
                tally["steps"] += int(st.sum())
                tally["runs"] += chunk
            j = (j + 1) % len(specs)

    oracle.lib()  # build/load before timing
    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker, args=(i,)) for i in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    sample = (f"{tally['runs']} runs ({tally['steps']} steps) drawn round-robin from the "
              f"{len(specs)} sets of the same workload, {dt:.1f} s wall on {threads} threads")
    return tally["steps"] / dt, threads, sample


def learned_bias_experiment(args, rates=None):
    """Learned bias vs the best constant bias on far-tail effective samples per
    second: m = 1, phi_in = 8, reflecting wall phi_uv = 9, dN = 5e-4, tail event
    N > 40, censored at N = 60.  A ladder of constant b (2^20 runs each) picks
    the best b by effective samples per EM step; that b is rerun on as many
    runs as the learned inference (2^26) for a like-for-like n_eff/s.  Training:
    --train-runs runs per Adam step (2^14), --train-steps steps (4096: 2^26 runs),
    timed on the host clock around the device-synchronised loop.  Everything
    is scaled by --scale.  The FP64 oracle runs the trained network on a
    bounded sample as a cross-check of the estimate.  Returns a dict."""
    import torch
    from paper_2206_11234_gb300 import native as nat
    from paper_2206_11234_gb300 import workloads as W
    import oracle
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    base = dict(phi_in=8.0, m=1.0, dN=5e-4, n_max=60.0, phi_uv=9.0)
    tail = 40.0
    p_ref = 1.0986e-3  # survival PDE (continuum limit)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b) / 1e3

    steps = torch.zeros(1, dtype=torch.int64, device=dev)

    def constant(b, n, seed):
        spec = W.SetSpec(n_traj=n, b=b, hist_lo=0.0, hist_hi=60.0, n_bins=512, **base)
        wl = W.Workload(f"const b={b}", [spec], "f32_f64acc", seed=seed)
        steps.zero_()
        (N, lw, _, _), t = timed(lambda: nat.simulate_workload(wl, with_hist=False, steps_out=steps))
        ne = tail_neff(N, lw, [spec], tail)[0]
        st = int(steps.item())
        return {"b": b, "runs": n, "P": ne["P"], "n_eff": ne["n_eff"], "seconds": t, "steps": st,
                "steps_per_s": st / t, "n_eff_per_s": ne["n_eff"] / t, "n_eff_per_Msteps": 1e6 * ne["n_eff"] / st}

    # the constant-bias runs take the library's autotuned launch shape (cached for
    # this precision, model and wall), as the main benchmark does
    pilot = W.SetSpec(n_traj=max(4096, int((1 << 22) * args.scale)), b=0.4, hist_lo=0.0, hist_hi=60.0, n_bins=512,
                      **base)
    tuned = nat.fpt_autotune(nat.make_params(precision="f32_f64acc", m=1.0, n_max=60.0, stream=stream),
                             nat.make_sets([pilot]), seed=99, fraction=0.02)
    n_c = max(4096, int((1 << 20) * args.scale))
    ladder = [constant(b, n_c, 11) for b in (0.0, 0.2, 0.4, 0.6, 0.8, 1.0, 2.0, 4.0, 6.0)]
    best_b = max(ladder, key=lambda r: r["n_eff_per_Msteps"])["b"]
    n_i = max(4096, int((1 << 26) * args.scale))
    with ClockSampler(0) as clk_c:
        best = constant(best_b, n_i, 13)
    # training, starting from the best constant amplitude
    n_t = max(1024, int(args.train_runs * args.scale))
    init = W.mlp_params(seed=5, gain=1.0, out_scale=0.05)
    init[-1] = best_b
    norm = (5.2, 0.5, 30.0, 1.0 / 15.0)
    tr = nat.MlpTrainer(W.SetSpec(n_traj=n_t, b=0.0, **base), init, norm, k_eval=args.k_eval, stream=stream)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.train_steps):
        hist.append(tr.step(seed=100000 + it, tail_N=tail, lr=args.lr))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # inference with the trained network
    spec = W.SetSpec(n_traj=n_i, b=0.0, **base)
    sets = nat.make_sets([spec])
    N = torch.empty(n_i, dtype=torch.float64, device=dev)
    lw = torch.empty(n_i, dtype=torch.float64, device=dev)
    p = nat.make_params(precision="f32_f64acc", m=1.0, n_max=60.0, mlp=tr.w, k_eval=args.k_eval, stream=stream,
                        steps_out=steps)
    warm = nat.make_sets([W.SetSpec(n_traj=min(n_i, 65536), b=0.0, **base)])
    nat.fpt_simulate_mlp(p, warm, 77, N, lw)  # warm-up
    steps.zero_()
    with ClockSampler(0) as clk_l:
        _, t_inf = timed(lambda: nat.fpt_simulate_mlp(p, sets, 12345, N, lw))
    ne = tail_neff(N, lw, [spec], tail)[0]
    st = int(steps.item())
    se_gpu = math.sqrt(max(ne["P"] ** 2 / max(ne["n_eff"], 1e-300), 0.0))
    learned = {"runs": n_i, "P": ne["P"], "se": se_gpu, "n_eff": ne["n_eff"], "seconds": t_inf, "steps": st,
               "steps_per_s": st / t_inf, "n_eff_per_s": ne["n_eff"] / t_inf,
               "n_eff_per_Msteps": 1e6 * ne["n_eff"] / st,
               "train_seconds": train_s, "train_runs": n_t * args.train_steps, "train_steps": args.train_steps,
               "rel_second_moment_log_first": hist[0]["log_second_moment"] - 2 * math.log(max(hist[0]["p_hat"], 1e-300)),
               "rel_second_moment_log_last": hist[-1]["log_second_moment"] - 2 * math.log(max(hist[-1]["p_hat"], 1e-300))}
    # roofline of the learned-bias stepper: the XU (MUFU) pipe binds, with the
    # constant-bias step's 3 operations per step plus 128 tanh per run every
    # k_eval steps; the tensor-core term is reported beside it
    pk = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    mufu_per_step = MUFU_PER_STEP + MLP_TANH_PER_EVAL / args.k_eval
    mufu_rate = learned["steps_per_s"] / 32 * mufu_per_step
    if rates:
        mufu_peak = rates["xu_lg2_per_s"] / 32
        src = "XU pipe measured in this run (fpt_pipe_rates: lg2.approx loop on every SM)"
    else:
        mufu_peak = n_sm * 0.5 * f_max
        src = f"{n_sm} SMs x 16 MUFU lanes/clk x {f_max / 1e6:.0f} MHz (max SM clock, MEASURED_PEAKS.json)"
    tflops = learned["steps_per_s"] * 2 * MLP_MAC_PER_EVAL / args.k_eval / 1e12
    bf16_peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
    roofline = {"bound": "alu", "achieved": mufu_rate / 1e9, "peak": mufu_peak / 1e9,
                "unit": "Gwarp-MUFU/s (algorithmic, XU pipe)", "frac": mufu_rate / mufu_peak, "traffic": None,
                "kernel": f"stepper_mlp_kernel<{args.k_eval}>", "mufu_per_warp_step": mufu_per_step,
                "peak_source": src,
                "tensor_term": {"achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s (bf16)",
                                "frac": tflops / bf16_peak if bf16_peak else None,
                                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS)"}}
    # FP64 oracle with the same (BF16) network on a bounded sample, all host cores
    p64 = nat.mlp_unpack_bf16(tr.master.cpu()).numpy()
    n_o = 1024
    res = [None] * 16

    def work(t):
        r = oracle.make_run(m=1.0, phi_in=8.0, phi_uv=9.0, dN=5e-4, n_max=60.0, seed=999, traj_offset=t * (n_o // 16),
                            mlp=p64, mlp_norm=norm, k_eval=args.k_eval)
        res[t] = oracle.simulate(r, n_o // 16)
    ths = [threading.Thread(target=work, args=(t,)) for t in range(16)]
    t0 = time.perf_counter()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    No = np.concatenate([r[0] for r in res])
    lo = np.concatenate([r[1] for r in res])
    xo = np.where(No > tail, np.exp(lo), 0.0)
    orc = {"runs": n_o, "P": float(xo.mean()), "se": float(xo.std() / math.sqrt(n_o)),
           "seconds": time.perf_counter() - t0}
    return {"event": f"N > {tail}", "reference_P_survival_pde": p_ref,
            "learned_vs_pde_rel": learned["P"] / p_ref - 1.0,
            "best_constant": best, "learned": learned, "oracle_learned": orc,
            "gain_n_eff_per_s": learned["n_eff_per_s"] / best["n_eff_per_s"] if best["n_eff_per_s"] else None,
            "roofline": roofline, "ladder": ladder,
            "constant_launch_shape": {"block_dim": tuned[0], "k_steps": tuned[1]},
            "k_eval": args.k_eval, "scale": args.scale, "lr": args.lr,
            "clocks": {"learned": clk_l.summary(), "best_constant": clk_c.summary()}}


def run_learned_bias(args):
    import torch
    from paper_2206_11234_gb300 import native as nat
    torch.cuda.set_device(0)
    rates = nat.fpt_pipe_rates()
    r = learned_bias_experiment(args, rates)
    L = r["learned"]
    line = {"metric": METRIC, "value": L["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * L["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "learned bias vs constant: m=1 phi_in=8 phi_uv=9 dN=5e-4, tail N > 40",
                       "scale": args.scale, "train_steps": args.train_steps, "lr": args.lr,
                       "k_eval": args.k_eval, "constant_launch_shape": r["constant_launch_shape"]},
            "clocks": r["clocks"]["learned"], "pipe_rates": rates,
            "tail": {k: r[k] for k in ("event", "reference_P_survival_pde", "best_constant", "learned",
                                       "oracle_learned", "gain_n_eff_per_s")},
            "roofline": r["roofline"], "ladder": r["ladder"]}
    print(json.dumps(line))


def run_estimators(args):
    """Per-bin estimators of §2.1 and §2.4 on simulated runs: the D'Agostino-
    Pearson test of ln w in each bin (>= 400 runs), the lognormal vs the direct
    estimate, jackknife vs analytic errors; drift-dominated (m = 0.01) and
    diffusion-dominated (m = 1, wall at 9) quadratic inflation, 2^20 runs per
    bias amplitude, 16 jackknife subsets; the estimate kernel timed alone."""
    import numpy as np
    import torch
    from paper_2206_11234_gb300 import native as nat
    from paper_2206_11234_gb300 import workloads as W
    n = max(1 << 14, int((1 << 20) * args.scale))
    n_sub = 16
    cases = [("drift m=0.01 phi_in=6 dN=1e-3", b, W.SetSpec(phi_in=6.0, m=0.01, b=b, dN=1e-3, n_max=10.0, n_traj=n,
                                                              hist_lo=8.45, hist_hi=8.85, n_bins=40))
             for b in (0.5, 1.0, 2.0, 4.0)]
    cases += [("diffusion m=1 phi_in=8 phi_uv=9 dN=5e-4", b,
               W.SetSpec(phi_in=8.0, m=1.0, b=b, dN=5e-4, n_max=60.0, phi_uv=9.0, n_traj=n, hist_lo=0.0,
                         hist_hi=60.0, n_bins=60)) for b in (0.4, 1.0)]
    rows = []
    kernel_ms = []
    for name, b, spec in cases:
        wl = W.Workload(name, [spec], "f32_f64acc", seed=4)
        N, lw, _, _ = nat.simulate_workload(wl, with_hist=False)
        bins = nat.empty_bins(spec.n_bins * n_sub)
        counts = nat.empty_counts(1)
        nat.fpt_histogram(N, lw, spec.n_bins, spec.hist_lo, spec.hist_hi, bins, counts, n_sub=n_sub)
        est = nat.empty_estimates(spec.n_bins)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        stream = torch.cuda.current_stream()
        for _ in range(3):
            nat.fpt_estimate(bins, spec.n_bins, spec.hist_lo, spec.hist_hi, n, est, n_sub=n_sub, stream=stream)
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(10):
            nat.fpt_estimate(bins, spec.n_bins, spec.hist_lo, spec.hist_hi, n, est, n_sub=n_sub, stream=stream)
        ev[1].record()
        torch.cuda.synchronize()
        kernel_ms.append(ev[0].elapsed_time(ev[1]) / 10)
        g = nat.estimates_to_dict(est)
        big = g["count"] >= 400
        p = g["p_normal"][big]
        d = np.abs(g["p_lognormal"][big] - g["p_direct"][big])
        err = np.hypot(np.maximum(g["eps_lo"][big], g["eps_hi"][big]), g["se_direct"][big])
        rows.append({"workload": name, "b": b, "bins_ge_400": int(big.sum()),
                     "p_normal_median": float(np.median(p)) if p.size else None,
                     "frac_p_below_0.005": float(np.mean(p < 0.005)) if p.size else None,
                     "lognormal_applies": nat.lognormal_applies(g),
                     "frac_lognormal_within_3sigma_of_direct": float(np.mean(d <= 3 * err)) if p.size else None,
                     "median_jk_over_se_direct": float(np.median(g["jk_direct"][big] / g["se_direct"][big]))
                     if p.size else None})
    print(json.dumps({"workload": "estimators", "runs_per_case": n, "n_sub": n_sub,
                      "estimate_kernel_ms": max(kernel_ms), "cases": rows}))


def run_power_bias(args):
    """The bias-optimisation experiment of §3.4: quadratic inflation m = 0.001,
    phi_in = 6 (drift domination), B = A_p phi^p for p = 0 .. 5 with A_p tuned
    so that the classical sample duration sits 8 classical sigma_N past the
    target's; dN = 1e-4 (sigma_N / 20); 2^18 runs per p (binary32 state,
    binary64 log-weight).  Scores each p by |r| of ln w with N (fpt_pearson) and
    by the relative errors of the direct and lognormal estimates in the bin at
    the sample mean."""
    import numpy as np
    import torch
    from paper_2206_11234_gb300 import native as nat
    from paper_2206_11234_gb300 import power_bias as PB
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m, phi_in, dN, shift = 1e-3, 6.0, 1e-4, 8.0
    n = max(1 << 12, int((1 << 18) * args.scale))
    sig = PB.classical_sigma(m, phi_in)
    n_t = PB.classical_duration(0.0, 1.0, phi_in)
    target = n_t + shift * sig
    N = torch.empty(n, dtype=torch.float64, device=dev)
    lw = torch.empty(n, dtype=torch.float64, device=dev)
    steps = torch.zeros(1, dtype=torch.int64, device=dev)
    rows = []
    for p in (0.0, 1.0, 2.0, 2.5, 3.0, 3.5, 4.0, 5.0):
        amp = PB.tune_amplitude(p, target, phi_in)
        prm = nat.make_params(precision="f32_f64acc", m=m, n_max=target + 40 * sig, bias_p=p, steps_out=steps)
        nat.fpt_simulate(prm, min(n, 4096), phi_in, PB.PHI_END, math.inf, dN, amp, 1, N, lw)  # warm-up
        steps.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        nat.fpt_simulate(prm, n, phi_in, PB.PHI_END, math.inf, dN, amp, 17, N, lw)
        ev[1].record()
        torch.cuda.synchronize()
        sec = ev[0].elapsed_time(ev[1]) / 1e3
        pr = nat.fpt_pearson(N, lw)
        # one bin of width sigma / 4 around the sample mean: relative errors of the two estimates
        lo = pr["mean_N"] - sig / 8
        bins = nat.empty_bins(1)
        counts = nat.empty_counts(1)
        nat.fpt_histogram(N, lw, 1, lo, lo + sig / 4, bins, counts)
        est = nat.empty_estimates(1)
        nat.fpt_estimate(bins, 1, lo, lo + sig / 4, n, est)
        e = nat.estimates_to_dict(est)
        st = int(steps.item())
        rows.append({"p": p, "A_p": amp, "abs_r": abs(pr["r"]), "mean_N": pr["mean_N"],
                     "mean_N_minus_target_in_sigma": (pr["mean_N"] - target) / sig,
                     "sd_lw": math.sqrt(pr["var_lw"]), "censored": n - int(pr["count"]),
                     "bin_runs": int(e["count"][0]),
                     "rel_err_direct": e["se_direct"][0] / e["p_direct"][0] if e["p_direct"][0] > 0 else None,
                     "rel_err_lognormal": e["eps_hi"][0] / e["p_lognormal"][0] if e["p_lognormal"][0] > 0 else None,
                     "p_normal": e["p_normal"][0], "steps_per_s": st / sec, "seconds": sec})
    best = max(rows, key=lambda r: r["abs_r"])
    print(json.dumps({"workload": "power_bias", "m": m, "phi_in": phi_in, "dN": dN, "runs_per_p": n,
                      "target_classical_N": n_t, "sigma_N": sig, "shift_sigmas": shift,
                      "best_p_by_abs_r": best["p"], "rows": rows}))


def run_multi_bias(args):
    """The multi-bias reconstruction of §3.2 (the paper's m = 0.1 experiment):
    quadratic inflation m = 0.1, phi_in = sqrt(42), no wall (censored at N = 20),
    dN = 1e-3, B = A S with A in {0, 0.5, ..., 3}, 2^20 runs per amplitude
    (binary32 state, binary64 log-weight); common bins on (9, 14] (width 0.025),
    20 jackknife subsets; per-bin lognormal estimates (bins with >= 400 runs and
    a normality p-value >= 0.5 %) stitched in log space (fpt_stitch).  Reports
    how deep the reconstruction reaches and whether overlapping amplitudes
    agree within their errors."""
    import numpy as np
    import torch
    from paper_2206_11234_gb300 import native as nat
    from paper_2206_11234_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = max(1 << 14, int((1 << 20) * args.scale))
    amps = (0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0)
    nb, lo, hi, n_sub = 200, 9.0, 14.0, 20
    specs = [W.SetSpec(phi_in=math.sqrt(42.0), m=0.1, b=a, dN=1e-3, n_max=20.0, n_traj=n, set_id=i, hist_lo=lo,
                       hist_hi=hi, n_bins=nb) for i, a in enumerate(amps)]
    wl = W.Workload("multi-bias", specs, "f32_f64acc", seed=3)
    steps = torch.zeros(1, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    nat.simulate_workload(W.Workload("warm", [W.SetSpec(**{**specs[0].__dict__, "n_traj": 4096})], "f32_f64acc"),
                          with_hist=False)
    torch.cuda.synchronize()
    ev[0].record()
    N, lw, _, _ = nat.simulate_workload(wl, with_hist=False, steps_out=steps)
    ev[1].record()
    torch.cuda.synchronize()
    sim_s = ev[0].elapsed_time(ev[1]) / 1e3
    est = torch.empty((len(amps), nb, len(nat.ESTIMATE_FIELDS)), dtype=torch.float64, device=dev)
    per = []
    for k, a in enumerate(amps):
        Nk, lk = N[k * n:(k + 1) * n].contiguous(), lw[k * n:(k + 1) * n].contiguous()
        bins = nat.empty_bins(nb * n_sub)
        counts = nat.empty_counts(1)
        nat.fpt_histogram(Nk, lk, nb, lo, hi, bins, counts, n_sub=n_sub, id_offset=k * n)
        nat.fpt_estimate(bins, nb, lo, hi, n, est[k], n_sub=n_sub, id_offset=k * n)
        fin = torch.isfinite(Nk)
        per.append({"A": a, "mean_N": Nk[fin].mean().item(), "censored": int((~fin).sum().item())})
    st = nat.fpt_stitch(est, estimator=nat.ESTIMATOR_LOGNORMAL, min_count=400, p_threshold=0.005).cpu().numpy()
    e = est.cpu().numpy()
    mid = lo + (np.arange(nb) + 0.5) * (hi - lo) / nb
    ok = np.isfinite(st[:, 0])
    # overlaps: every pair of contributing amplitudes in a bin within 4 combined errors
    pairs = agree = 0
    for j in np.nonzero(st[:, 4] >= 2)[0]:
        use = []
        for k in range(len(amps)):
            c, pn, v = e[k, j, 0], e[k, j, 13], e[k, j, 7]
            if c >= 400 and (pn >= 0.005 or v == 0) and e[k, j, 3] > 0:
                use.append((math.log(e[k, j, 3]), math.sqrt(v / c + v * v / (2 * c - 2) + 1 / c)))
        for x in range(len(use)):
            for y in range(x + 1, len(use)):
                pairs += 1
                agree += abs(use[x][0] - use[y][0]) <= 4 * math.hypot(use[x][1], use[y][1])
    for k, r in enumerate(per):
        use = (e[k, :, 0] >= 400) & ((e[k, :, 13] >= 0.005) | (e[k, :, 7] == 0)) & (e[k, :, 3] > 0)
        r["bins_used"] = int(use.sum())
        r["N_range"] = [float(mid[use].min()), float(mid[use].max())] if use.any() else None
        r["min_P"] = float(e[k, use, 3].min()) if use.any() else None
    line = {"workload": "multi_bias", "m": 0.1, "phi_in": math.sqrt(42.0), "dN": 1e-3, "runs_per_amplitude": n,
            "total_runs": n * len(amps), "steps": int(steps.item()), "simulate_seconds": sim_s,
            "steps_per_s": int(steps.item()) / sim_s, "per_amplitude": per,
            "stitched": {"bins": int(ok.sum()), "N_max": float(mid[ok].max()), "min_P": float(st[ok, 0].min()),
                         "max_rel_err": float(st[ok, 3].max()), "median_rel_err": float(np.median(st[ok, 3]))},
            "overlap_pairs": pairs, "overlap_agree_4sigma": agree / pairs if pairs else None,
            "curve": [[float(x), float(p), float(a)] for x, p, a in zip(mid[ok][::10], st[ok, 0][::10], st[ok, 3][::10])]}
    print(json.dumps(line))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload, args.scale)
    per = max(args.cpu_seconds / max(args.steps, 1), 1.0)
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, min(per, 2.0))
    rates = []
    t0 = time.perf_counter()
    cores = 1
    sample = ""
    for _ in range(args.steps):
        r, cores, sample = cpu_oracle_rate(wl, per)
        rates.append(r)
    total_t = time.perf_counter() - t0
    v = statistics.mean(rates)
    line = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "precision": "f64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "learned_bias":
        return run_learned_bias(args)
    if args.workload == "estimators":
        return run_estimators(args)
    if args.workload == "power_bias":
        return run_power_bias(args)
    if args.workload == "multi_bias":
        return run_multi_bias(args)

    import torch
    import torch.distributed as dist
    from paper_2206_11234_gb300 import native as nat
    from paper_2206_11234_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    # measured pipe rates of this GPU (the denominators of the rooflines below)
    rates = nat.fpt_pipe_rates()
    wl = make_workload(args.workload, args.scale)
    # weak scaling: each rank simulates its own disjoint id range of every set
    for s in wl.sets:
        s.traj_offset = rank * s.n_traj
    specs = wl.sets
    n = wl.n_total
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    N = torch.empty(n, dtype=torch.float64, device=dev)
    lw = torch.empty(n, dtype=torch.float64, device=dev)
    nbins = sum(s.n_bins for s in specs)
    bins = nat.empty_bins(nbins, dev)
    counts = nat.empty_counts(len(specs), dev)
    steps_ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    sets = nat.make_sets(specs)
    s0 = specs[0]

    def params(prec, steps_out=None):
        return nat.make_params(model=s0.model, precision=prec, m=s0.m, a0=s0.a0, s0=s0.s0,
                               n_max=s0.n_max, block_dim=args.block_dim, k_steps=args.k_steps,
                               stream=stream, steps_out=steps_out)

    # launch shape from the library's autotuner (pilot on 2 % of the workload; untimed setup)
    tuned = None
    if args.block_dim == 0 and args.k_steps == 0:
        tb, tk, trate = nat.fpt_autotune(params(wl.precision), sets, seed=99, fraction=0.02)
        tuned = {"block_dim": tb, "k_steps": tk, "pilot_steps_per_s": trate}
    p = params(wl.precision, steps_ctr)
    # one graph-captured launch per step: stepper over all sets + histograms
    plan = nat.Plan(p, sets, N, lw, bins, counts)
    plan_stepper = nat.Plan(p, sets, N, lw)

    def one_step(seed):
        plan.launch(seed, stream)

    # L2: every step writes its outputs (16 B per run).  When they do not
    # exceed twice the L2, a buffer of twice the L2 is rewritten before each
    # timed step, outside the timed events
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (129 << 20))
    flush = torch.empty(2 * l2_bytes // 4, dtype=torch.int32, device=dev) if 16 * n < 2 * l2_bytes else None

    def timed_steps(launch):
        """ms over args.steps launches, with the L2 flushed between them if needed."""
        if flush is None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(args.steps):
                launch(i)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)
        evs = []
        for i in range(args.steps):
            flush.fill_(i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            launch(i)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    for i in range(args.warmup):
        one_step(1000 + i)
    torch.cuda.synchronize()
    steps_ctr.zero_()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed_steps(one_step)
    if world > 1:
        dist.barrier()
    my_steps = int(steps_ctr.item())
    t = torch.tensor([ms, float(my_steps)], dtype=torch.float64, device=dev)
    if world > 1:
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms_max, total_steps = tmax[0].item(), tsum[1].item()
    else:
        ms_max, total_steps = ms, float(my_steps)
    value = total_steps / (ms_max / 1e3)

    # the per-rank histograms of the last timed step merged into the histogram of
    # the whole job (gather over the process group, fpt_hist_merge on the host;
    # the counters are integers and add): outside the timed region
    hist_merge = None
    if world > 1:
        from paper_2206_11234_gb300 import shard
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        merged_bins, _ = shard.allgather_merge(bins)
        merged_counts = counts.clone()
        dist.all_reduce(merged_counts, op=dist.ReduceOp.SUM)
        hist_merge = {"ranks": world, "bins": nbins, "seconds": time.perf_counter() - t0,
                      "runs": int(merged_counts[:, 3].sum().item()),
                      "in_range": int(merged_bins.numpy().view(np.int64)[:, 7].sum())}

    # the stepper kernel alone (CUDA events on the launching stream), for the roofline
    ms_stepper = None
    if rank == 0:
        steps_ctr.zero_()
        torch.cuda.synchronize()
        ms_stepper = timed_steps(lambda i: plan_stepper.launch(i, stream)) / args.steps
        stepper_steps = int(steps_ctr.item()) / args.steps

    extra = {}
    if hist_merge is not None:
        extra["hist_merge"] = hist_merge
    if rank == 0:
        # far-tail effective samples (E = {N > tail_N}) of the last timed step's runs
        plan.launch(args.steps - 1, stream)
        if wl.tail_N is not None:
            ne = tail_neff(N, lw, specs, wl.tail_N)
            # each set's share of the step time: its EM steps (from the records: the
            # crossing step ceil(N/dN), or the cap ceil(n_max/dN) when censored) over all
            t_step = ms_max / 1e3 / args.steps
            off = 0
            for s_, r_ in zip(specs, ne):
                Ns = N[off:off + s_.n_traj]
                cap = float(math.ceil(s_.n_max / s_.dN))
                r_["steps"] = torch.where(torch.isfinite(Ns), torch.ceil(Ns / s_.dN), torch.full_like(Ns, cap)).sum().item()
                off += s_.n_traj
            tot = sum(r_["steps"] for r_ in ne) or 1.0
            for r_ in ne:
                r_["seconds"] = t_step * r_["steps"] / tot
                r_["n_eff_per_s"] = r_["n_eff"] / r_["seconds"] if r_["seconds"] > 0 else 0.0
            best = max(ne, key=lambda r: r["n_eff_per_s"])
            extra["tail"] = {"event": f"N > {wl.tail_N}", "per_set": ne,
                             "best_n_eff_per_s": best["n_eff_per_s"], "best_b": best["b"],
                             "time_share": "each set's n_eff over its share of the step time (its EM steps / all)"}
    # end to end through the host-buffer entry (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hN = torch.empty(n, dtype=torch.float64).pin_memory()
        hl = torch.empty(n, dtype=torch.float64).pin_memory()
        hb = torch.empty((nbins, nat.BIN_FIELDS), dtype=torch.float64).pin_memory()
        hc = torch.empty((len(specs), 4), dtype=torch.int64).pin_memory()
        pe = params(wl.precision, steps_ctr)
        nat.fpt_simulate_batch_host(pe, sets, 7, hN, hl, hb, hc)
        steps_ctr.zero_()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk_e:
            # host-timed: let nvidia-smi start and take its first sample (its
            # start-up can hold up this process's CUDA calls) before the clock starts
            time.sleep(0.5)
            t0 = time.perf_counter()
            for i in range(args.steps):
                nat.fpt_simulate_batch_host(pe, sets, i, hN, hl, hb, hc)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        tt = torch.tensor([dt, float(steps_ctr.item())], dtype=torch.float64, device=dev)
        if world > 1:
            t1 = tt.clone()
            dist.all_reduce(t1, op=dist.ReduceOp.MAX)
            t2 = tt.clone()
            dist.all_reduce(t2, op=dist.ReduceOp.SUM)
            dt, es = t1[0].item(), t2[1].item()
        else:
            es = tt[1].item()
        # the link's own rate for the record copies on this machine (outside the
        # timed loop): the part of a call that overlapping can hide
        torch.cuda.synchronize()
        tl = time.perf_counter()
        for _ in range(3):
            hN.copy_(N, non_blocking=True)
            hl.copy_(lw, non_blocking=True)
        torch.cuda.synchronize()
        link_s = (time.perf_counter() - tl) / 3
        import ctypes
        h2d = ctypes.sizeof(nat.FptSet) * len(specs) + ctypes.sizeof(nat.FptParams)
        d2h = 2 * 8 * n + ctypes.sizeof(nat.FptBin) * nbins + ctypes.sizeof(nat.FptHistCounts) * len(specs)
        e2e = {"value": es / dt, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_call": dt / args.steps * 1e3,
               "records_d2h_ms": link_s * 1e3, "records_d2h_gbs": 16 * n / link_s / 1e9,
               "copies": "records on a second stream during the histogram kernels, then bins and counters",
               "clocks": clk_e.summary()}

    # FP64 GPU plain on a bounded sample of the same workload (speed reference),
    # after the end-to-end loop, which runs in the state the device-timed steps
    # left (on the 64-set workload the loop measured 4.6 % above the device step
    # when it ran after this sample, 1.2 % without it)
    if rank == 0 and not args.no_f64:
        frac = min(1.0, 2**16 * len(specs) / n)
        wl64 = make_workload(args.workload, args.scale * frac)
        p64 = nat.make_params(model=s0.model, precision="f64", m=s0.m, a0=s0.a0, s0=s0.s0, n_max=s0.n_max,
                              block_dim=256, k_steps=4, stream=stream, steps_out=steps_ctr)
        n64 = wl64.n_total
        N64 = torch.empty(n64, dtype=torch.float64, device=dev)
        l64 = torch.empty(n64, dtype=torch.float64, device=dev)
        s64 = nat.make_sets(wl64.sets)
        nat.fpt_simulate_batch(p64, s64, 0, N64, l64, None, None)
        steps_ctr.zero_()
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nat.fpt_simulate_batch(p64, s64, 1, N64, l64, None, None)
        b_.record(stream)
        torch.cuda.synchronize()
        st64 = int(steps_ctr.item())
        extra["f64_gpu_plain"] = {"value": st64 / (a.elapsed_time(b_) / 1e3), "unit": "steps/s", "runs": n64,
                                  "steps": st64, "block_dim": 256, "k_steps": 4}
        del N64, l64

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    # three pipes bound the binary32 step: instruction issue (1 per SM
    # sub-partition per clock), the XU pipe (MUFU) and the fma-heavy pipe (the
    # Philox wide multiplies); the XU and wide-multiply peaks are measured in
    # this run by the library's pipe-rate loops (thread operations per second)
    issue_peak = n_sm * ISSUE_PER_SM_CLK * f_max           # warp-instructions/s
    mufu_peak = rates["xu_lg2_per_s"] / 32                  # warp-MUFU/s
    wide_peak = rates["wide_mul_per_s"] / 32                # warp wide multiplies/s
    bounds = {"issue": issue_peak / ALG_INST_PER_STEP * 32, "xu": mufu_peak / MUFU_PER_STEP * 32,
              "fma_heavy": wide_peak / WIDE_MUL_PER_STEP * 32}
    binding = min(bounds, key=bounds.get)
    steps_peak = bounds[binding]
    achieved_steps = stepper_steps / (ms_stepper / 1e3)
    shape = tuned or {"block_dim": args.block_dim, "k_steps": args.k_steps}
    ctr = stepper_counters(wl.precision, shape.get("block_dim"), shape.get("k_steps"))
    measured = None
    if ctr:
        ws = ctr["steps"] / 32.0
        inst_ws = ctr["inst_executed"] / ws  # warp-instructions per warp-step
        measured = {"inst_per_warp_step": inst_ws,
                    "steps_per_s_peak": issue_peak / inst_ws * 32,
                    "frac": achieved_steps / (issue_peak / inst_ws * 32),
                    "xu_inst_per_warp_step": ctr.get("inst_xu", 0) / ws,
                    "fma_heavy_cycles_per_warp_step": ctr.get("fmaheavy_cycles", 0) / (4 * n_sm) / (ws / (4 * n_sm)),
                    "pipe_busy_pct": ctr.get("pipe_busy_pct"),
                    "branch_targets_uniform_pct": ctr["branch_targets_uniform_pct"],
                    "active_lanes_per_inst_pct": 100.0 * ctr["thread_inst_executed"] / (32.0 * ctr["inst_executed"]),
                    "source": "profiles/stepper_counters.json"}
    units = {"issue": ("Gwarp-inst/s (algorithmic)", ALG_INST_PER_STEP, issue_peak),
             "xu": ("Gwarp-MUFU/s (algorithmic, XU pipe)", MUFU_PER_STEP, mufu_peak),
             "fma_heavy": ("Gwarp-wide-multiplies/s (algorithmic, fma-heavy pipe)", WIDE_MUL_PER_STEP, wide_peak)}

    def term(name):
        u, per, pk_ = units[name]
        return {"achieved": achieved_steps * per / 32 / 1e9, "peak": pk_ / 1e9, "unit": u,
                "frac": achieved_steps / bounds[name], "per_warp_step": per, "steps_per_s_bound": bounds[name]}
    u_, per_, p_ = units[binding]
    roof = {"bound": "alu", "binding_pipe": binding, "achieved": achieved_steps * per_ / 32 / 1e9, "peak": p_ / 1e9,
            "unit": u_, "frac": achieved_steps / steps_peak,
            "issue_term": term("issue"), "xu_term": term("xu"), "fma_heavy_term": term("fma_heavy"),
            "traffic": (ctr["dram_read_bytes"] + ctr["dram_write_bytes"]) * n / ctr["runs"] if ctr else None,
            "vs_measured_instructions": measured,
            "kernel": f"stepper_kernel<float, {wl.precision}, quadratic, "
                      f"block_dim {shape.get('block_dim')}, k_steps {shape.get('k_steps')}>",
            "steps_per_s": achieved_steps, "steps_per_s_peak": steps_peak,
            "peak_source": (f"issue: {n_sm} SMs x 4 issue/clk x {f_max / 1e6:.0f} MHz (max SM clock, "
                            "MEASURED_PEAKS.json); XU and fma-heavy: measured in this run by fpt_pipe_rates "
                            "(one-instruction loops on every SM)")}
    if wl.precision == "f64":
        # the binary64 reference path (per-run parity configuration)
        roof = {"bound": "fp64", "achieved": achieved_steps, "peak": None, "unit": "steps/s", "frac": None,
                "traffic": None, "kernel": f"stepper_kernel<double, f64, {wl.sets[0].model and 'constant' or 'quadratic'}, "
                                           f"k_steps {shape.get('k_steps')}>",
                "note": "binary64 reference path: its FP64-pipe fraction is in f64_gpu_plain.roofline of the "
                        "binary32 workloads' lines"}
    if "f64_gpu_plain" in extra:
        # FP64 roofline: FP64-pipe warp-instructions per warp-step (ncu record of the
        # binary64 stepper) x the live rate, against the measured DFMA rate
        f64 = extra["f64_gpu_plain"]
        c64 = stepper_counters("f64", f64.get("block_dim"), f64.get("k_steps"), name="stepper_f64_counters.json")
        fp64_peak = rates["fp64_fma_per_s"] / 32  # warp DFMA/s
        if c64:
            ws64 = c64["steps"] / 32.0
            per = c64["inst_fp64"] / ws64
            ach = f64["value"] / 32 * per
            # the FP64 pipe's busy fraction at the live rate: its ncu cycles per
            # warp-step (per SM) x warp-steps per second and SM / clock
            busy = f64["value"] / 32 / n_sm * (c64["fp64_pipe_cycles"] / ws64) / f_max
            f64["roofline"] = {"bound": "fp64", "achieved": ach / 1e9, "peak": fp64_peak / 1e9,
                               "unit": "Gwarp-FP64-inst/s", "frac": ach / fp64_peak,
                               "fp64_inst_per_warp_step": per, "steps_per_s_bound": fp64_peak / per * 32,
                               "fp64_pipe_busy_live": busy, "pipe_busy_pct_ncu": c64.get("fp64_pipe_busy_pct"),
                               "peak_source": "DFMA loop on every SM in this run (fpt_pipe_rates); the stepper's "
                                              "FP64 instructions also include cheaper ones, so frac can pass 1",
                               "source": "profiles/stepper_f64_counters.json"}
        else:
            f64["roofline"] = {"bound": "fp64", "peak": fp64_peak / 1e9, "unit": "Gwarp-DFMA/s", "frac": None,
                               "note": "no ncu record of the FP64-pipe instructions for this kernel and shape"}
    cpu = None
    if not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl, args.cpu_seconds)
        rate1, _, sample1 = cpu_oracle_rate(wl, min(3.0, args.cpu_seconds), threads=1)
        cpu = {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": rate1, "sample": sample1}}
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl.precision != "f64" else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "precision": wl.precision, "runs_per_gpu": n,
                   "em_steps_per_step": total_steps / args.steps,
                   "sets": len(specs),
                   "l2": (f"outputs (16 B/run, {16 * n / 2**20:.0f} MiB) exceed L2 ({l2_bytes / 2**20:.0f} MiB); "
                          "no inputs besides parameters" if flush is None else
                          f"outputs ({16 * n / 2**20:.1f} MiB) fit in L2 ({l2_bytes / 2**20:.0f} MiB): a "
                          f"{2 * l2_bytes / 2**20:.0f} MiB buffer is rewritten before each timed step, outside "
                          "the timed events"),
                   "parallelism": f"dp{world} (disjoint run ids per GPU)",
                   "launch_shape": tuned or {"block_dim": args.block_dim, "k_steps": args.k_steps}},
        "gpu_launches": 5 * args.steps,
        "launch": "one CUDA graph per step (fpt_plan: scratch reset, stepper, 4 histogram kernels)",
        "clocks": clk.summary(),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "context": "the paper's CPU package (Python) reports ~8 h for 2e5 drift-dominated runs on a quad-core "
                   "laptop and 'a few hours on a single CPU' for the whole study; it gives no steps/s",
    }
    line["pipe_rates"] = dict(rates, per_sm_clock={k: v / (n_sm * f_max) for k, v in rates.items()},
                              clock_assumed_mhz=f_max / 1e6)
    line.update(extra)
    if world == 1 and args.workload == "drift_ladder" and not args.no_learned:
        # the learned-bias configuration (m = 1, phi_in = 8, wall 9, tail N > 40):
        # learned vs best constant bias on far-tail effective samples per second
        line["learned_bias"] = learned_bias_experiment(args, rates)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
