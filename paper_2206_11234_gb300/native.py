"""Thin ctypes binding of the C ABI in include/fpt.h (argument marshalling only).

Every function forwards to the CUDA library libfpt_gb300.so; there is no
fallback: if the library is missing or cannot be loaded, importing this module
raises.  Device arrays are torch CUDA tensors (torch provides device memory and
streams); their data pointers are passed through unchanged.
"""
import ctypes
import math
import os
from typing import List, Optional, Sequence

import torch

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))

FPT_ABI_VERSION = 3
FPT_OK = 0
FPT_EINVAL = -1
FPT_ECUDA = -2
FPT_ENOMEM = -3
FPT_EUNSUPPORTED = -4
FPT_EDEVICE_STATUS = -5

MODEL_QUADRATIC = 0
MODEL_CONSTANT = 1
MODEL_POLYNOMIAL = 2
POLY_TERMS = 8
PREC_F64 = 0
PREC_F32_KAHAN = 1
PREC_F32_F64ACC = 2
PRECISIONS = {"f64": PREC_F64, "f32_kahan": PREC_F32_KAHAN, "f32_f64acc": PREC_F32_F64ACC}
BIAS_CONST = 0
BIAS_POWER = 1
BIAS_MLP = 2
MAX_SETS = 64
MAX_HIST_BINS = 4096


class FptParams(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32),
        ("model", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("bias_kind", ctypes.c_int32),
        ("m", ctypes.c_double),
        ("a0", ctypes.c_double),
        ("s0", ctypes.c_double),
        ("n_max", ctypes.c_double),
        ("bias_p", ctypes.c_double),
        ("poly", ctypes.c_double * 8),
        ("mlp", ctypes.c_void_p),
        ("k_eval", ctypes.c_int32),
        ("block_dim", ctypes.c_int32),
        ("k_steps", ctypes.c_int32),
        ("set_id", ctypes.c_uint32),
        ("traj_offset", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("steps_out", ctypes.c_void_p),
    ]


class FptPipeRates(ctypes.Structure):
    _fields_ = [
        ("fp64_fma_per_s", ctypes.c_double),
        ("xu_lg2_per_s", ctypes.c_double),
        ("wide_mul_per_s", ctypes.c_double),
        ("fp32_fma_per_s", ctypes.c_double),
    ]


class FptSet(ctypes.Structure):
    _fields_ = [
        ("phi_in", ctypes.c_double),
        ("phi_end", ctypes.c_double),
        ("phi_uv", ctypes.c_double),
        ("m", ctypes.c_double),
        ("b", ctypes.c_double),
        ("dN", ctypes.c_double),
        ("n_max", ctypes.c_double),
        ("n_traj", ctypes.c_int64),
        ("traj_offset", ctypes.c_uint64),
        ("set_id", ctypes.c_uint32),
        ("n_bins", ctypes.c_int32),
        ("hist_lo", ctypes.c_double),
        ("hist_hi", ctypes.c_double),
    ]


class FptBin(ctypes.Structure):
    _fields_ = [("max_lw", ctypes.c_double), ("s1", ctypes.c_double), ("s2", ctypes.c_double),
                ("l1", ctypes.c_double), ("l2", ctypes.c_double), ("l3", ctypes.c_double),
                ("l4", ctypes.c_double), ("count", ctypes.c_int64)]


ESTIMATE_FIELDS = ("count", "p_direct", "se_direct", "p_lognormal", "eps_lo", "eps_hi", "mean_lw", "var_lw",
                   "skew", "kurt", "z_skew", "z_kurt", "k2", "p_normal", "jk_direct", "jk_lognormal",
                   "bias_ln", "bias_se")


class FptEstimateBin(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in ESTIMATE_FIELDS]


class FptHistCounts(ctypes.Structure):
    _fields_ = [("under", ctypes.c_int64), ("over", ctypes.c_int64), ("censored", ctypes.c_int64),
                ("total", ctypes.c_int64)]


class FptMlpTrainState(ctypes.Structure):
    _fields_ = [("master", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("w", ctypes.c_void_p), ("records", ctypes.c_void_p),
                ("record_capacity", ctypes.c_int64), ("out_N", ctypes.c_void_p), ("out_logw", ctypes.c_void_p),
                ("coef", ctypes.c_void_p), ("rows", ctypes.c_void_p), ("step", ctypes.c_int32)]


class FptMlpTrainStats(ctypes.Structure):
    _fields_ = [("log_second_moment", ctypes.c_double), ("p_hat", ctypes.c_double), ("n_eff", ctypes.c_double),
                ("frac_in_tail", ctypes.c_double), ("n_records", ctypes.c_int64)]


BIN_FIELDS = 8  # an fpt_bin is 8 x 8 bytes: view bins as float64[n, 8] (count as int64 bits)


class FptError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


# FPT_DEBUG_LIB=1: load the build with device bounds checks (build.py --debug)
DEBUG_LIB = os.environ.get("FPT_DEBUG_LIB", "0") == "1"


def _load():
    path = _build.lib_path(DEBUG_LIB)
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2206_11234_gb300/build.py "
                          "(python -c 'import __graft_entry__ as g; g.build()'" +
                          (", or build.py --debug for the checked build)" if DEBUG_LIB else ")"))
    if not _build.up_to_date(DEBUG_LIB):
        raise ImportError(f"{path} is older than its sources: rebuild it")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, d, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_uint32, ctypes.c_uint64)
    L.fpt_simulate.argtypes = [P(FptParams), i64, d, d, d, d, d, u64, vp, vp]
    L.fpt_simulate_batch.argtypes = [P(FptParams), P(FptSet), i32, u64, vp, vp, vp, vp]
    L.fpt_simulate_batch_host.argtypes = [P(FptParams), P(FptSet), i32, u64, vp, vp, vp, vp]
    L.fpt_histogram.argtypes = [vp, vp, i64, i32, d, d, i32, u64, vp, vp, vp]
    L.fpt_estimate.argtypes = [vp, i32, i32, d, d, i64, u64, vp, vp]
    L.fpt_pearson.argtypes = [vp, vp, i64, vp, vp]
    L.fpt_stitch.argtypes = [vp, i32, i32, i32, i64, d, vp, vp]
    L.fpt_normals.argtypes = [u64, u64, u32, u32, i64, i32, vp, vp]
    L.fpt_autotune.argtypes = [P(FptParams), P(FptSet), i32, u64, d, P(i32), P(i32), P(d)]
    L.fpt_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp]
    L.fpt_simulate_mlp.argtypes = [P(FptParams), P(FptSet), i32, u64, vp, vp, vp, i64, P(i64)]
    L.fpt_plan_create.argtypes = [P(FptParams), P(FptSet), i32, vp, vp, vp, vp, P(vp)]
    L.fpt_plan_launch.argtypes = [vp, u64, vp]
    L.fpt_plan_destroy.argtypes = [vp]
    L.fpt_mlp_train_step.argtypes = [P(FptParams), P(FptSet), u64, d, d, P(FptMlpTrainState),
                                     P(FptMlpTrainStats)]
    L.fpt_mlp_backward.argtypes = [vp, vp, vp, vp, i64, vp, vp]
    L.fpt_wait_selftest.argtypes = [P(i32), P(d), vp]
    L.fpt_wait_selftest.restype = ctypes.c_int
    L.fpt_inject_alloc_failures.argtypes = [i32]
    L.fpt_inject_alloc_failures.restype = ctypes.c_int
    L.fpt_inject_status.argtypes = [u32]
    L.fpt_inject_status.restype = ctypes.c_int
    L.fpt_hist_merge.argtypes = [vp, i32, i64, vp, vp, vp]
    L.fpt_hist_merge.restype = ctypes.c_int
    L.fpt_pipe_rates.argtypes = [P(FptPipeRates), vp]
    L.fpt_pipe_rates.restype = ctypes.c_int
    L.fpt_autotune_reset.argtypes = []
    L.fpt_autotune_reset.restype = None
    L.fpt_strerror.restype = ctypes.c_char_p
    L.fpt_strerror.argtypes = [ctypes.c_int]
    L.fpt_last_error.restype = ctypes.c_char_p
    L.fpt_abi_version.restype = ctypes.c_int
    for name in ("fpt_simulate", "fpt_simulate_batch", "fpt_simulate_batch_host", "fpt_histogram",
                 "fpt_normals", "fpt_autotune", "fpt_mlp_forward", "fpt_mlp_backward", "fpt_simulate_mlp",
                 "fpt_mlp_train_step", "fpt_plan_create", "fpt_plan_launch", "fpt_plan_destroy"):
        getattr(L, name).restype = ctypes.c_int
    if L.fpt_abi_version() != FPT_ABI_VERSION:
        raise ImportError("libfpt_gb300.so ABI version mismatch")
    return L


lib = _load()


def _check(rc):
    if rc != FPT_OK:
        raise FptError(rc, f"{lib.fpt_strerror(rc).decode()}: {lib.fpt_last_error().decode()}")


def _dptr(t: Optional[torch.Tensor], dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_params(*, model=MODEL_QUADRATIC, precision=PREC_F64, m=1.0, a0=0.0, s0=0.0, n_max,
                block_dim=0, k_steps=0, set_id=0, traj_offset=0, stream=None,
                steps_out: Optional[torch.Tensor] = None, mlp: Optional[torch.Tensor] = None,
                k_eval: int = 0, bias_p: Optional[float] = None, poly=None) -> FptParams:
    """Launch parameters.  The bias is B = b S (the sets' b) by default, the
    power law B = b phi^bias_p when bias_p is given, the learned b(phi, N) S
    when mlp is given.  poly: coefficients c_0.. of V = sum_k c_k phi^k for
    model=MODEL_POLYNOMIAL (at most POLY_TERMS)."""
    p = FptParams()
    p.abi_version = FPT_ABI_VERSION
    p.model = model
    p.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    p.bias_kind = BIAS_CONST if mlp is None else BIAS_MLP
    if bias_p is not None:
        if mlp is not None:
            raise ValueError("bias_p and mlp exclude each other")
        p.bias_kind = BIAS_POWER
        p.bias_p = bias_p
    p.m, p.a0, p.s0, p.n_max = m, a0, s0, n_max
    if poly is not None:
        c = [float(x) for x in poly]
        if len(c) > POLY_TERMS:
            raise ValueError(f"at most {POLY_TERMS} coefficients")
        p.poly = (ctypes.c_double * POLY_TERMS)(*(c + [0.0] * (POLY_TERMS - len(c))))
    p.mlp = None if mlp is None else mlp.data_ptr()
    p.k_eval = k_eval
    p.block_dim, p.k_steps = block_dim, k_steps
    p.set_id, p.traj_offset = set_id, traj_offset
    p.stream = _stream(stream)
    p.steps_out = None if steps_out is None else steps_out.data_ptr()
    return p


def fpt_simulate(params: FptParams, n_traj: int, phi_in: float, phi_end: float, phi_uv: float,
                 dN: float, bias: float, seed: int, out_N: torch.Tensor, out_logw: torch.Tensor):
    _check(lib.fpt_simulate(ctypes.byref(params), n_traj, phi_in, phi_end, phi_uv, dN, bias, seed,
                            _dptr(out_N, torch.float64), _dptr(out_logw, torch.float64)))


def make_sets(specs: Sequence) -> ctypes.Array:
    """fpt_set[] from objects with the fields of workloads.SetSpec."""
    arr = (FptSet * len(specs))()
    off = 0
    for i, s in enumerate(specs):
        a = arr[i]
        a.phi_in, a.phi_end, a.phi_uv = s.phi_in, s.phi_end, s.phi_uv
        a.m, a.b, a.dN, a.n_max = s.m, s.b, s.dN, s.n_max
        a.n_traj = s.n_traj
        a.traj_offset = getattr(s, "traj_offset", 0)
        a.set_id = s.set_id
        a.n_bins = s.n_bins
        a.hist_lo, a.hist_hi = s.hist_lo, s.hist_hi
        off += s.n_traj
    return arr


def fpt_simulate_batch(params: FptParams, sets: ctypes.Array, seed: int, out_N: torch.Tensor,
                       out_logw: torch.Tensor, out_bins: Optional[torch.Tensor] = None,
                       out_counts: Optional[torch.Tensor] = None):
    _check(lib.fpt_simulate_batch(ctypes.byref(params), sets, len(sets), seed,
                                  _dptr(out_N, torch.float64), _dptr(out_logw, torch.float64),
                                  _dptr(out_bins), _dptr(out_counts)))


class Plan:
    """A graph-captured batched launch (fpt_plan_*) writing into fixed device tensors."""

    def __init__(self, params: FptParams, sets: ctypes.Array, out_N: torch.Tensor, out_logw: torch.Tensor,
                 out_bins: Optional[torch.Tensor] = None, out_counts: Optional[torch.Tensor] = None):
        self._keep = (sets, out_N, out_logw, out_bins, out_counts)
        h = ctypes.c_void_p()
        _check(lib.fpt_plan_create(ctypes.byref(params), sets, len(sets), _dptr(out_N, torch.float64),
                                   _dptr(out_logw, torch.float64), _dptr(out_bins), _dptr(out_counts),
                                   ctypes.byref(h)))
        self.handle = h

    def launch(self, seed: int, stream=None):
        _check(lib.fpt_plan_launch(self.handle, seed, _stream(stream)))

    def close(self):
        if self.handle:
            lib.fpt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fpt_simulate_batch_host(params: FptParams, sets: ctypes.Array, seed: int, host_N, host_logw,
                            host_bins, host_counts):
    """Host buffers: torch CPU tensors (pinned or not), or None for N/logw."""
    def hp(t):
        if t is None:
            return None
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return ctypes.c_void_p(t.data_ptr())
    _check(lib.fpt_simulate_batch_host(ctypes.byref(params), sets, len(sets), seed, hp(host_N),
                                       hp(host_logw), hp(host_bins), hp(host_counts)))


def fpt_histogram(N: torch.Tensor, logw: torch.Tensor, n_bins: int, lo: float, hi: float,
                  bins: torch.Tensor, counts: torch.Tensor, n_sub: int = 1, id_offset: int = 0,
                  stream=None):
    _check(lib.fpt_histogram(_dptr(N, torch.float64), _dptr(logw, torch.float64), N.numel(), n_bins,
                             lo, hi, n_sub, id_offset, _dptr(bins), _dptr(counts), _stream(stream)))


def fpt_estimate(bins: torch.Tensor, n_bins: int, lo: float, hi: float, n_total: int, out: torch.Tensor,
                 n_sub: int = 1, id_offset: int = 0, stream=None):
    """Per-bin estimates (fpt_estimate_bin, viewed as float64[n_bins, 16]) of a
    histogram of n_total runs; `bins` as written by fpt_histogram."""
    if out.dtype != torch.float64 or out.numel() < 16 * n_bins:
        raise ValueError("out must be float64 with 16 values per bin")
    _check(lib.fpt_estimate(_dptr(bins), n_bins, n_sub, lo, hi, n_total, id_offset, _dptr(out),
                            _stream(stream)))


ESTIMATOR_DIRECT = 0
ESTIMATOR_LOGNORMAL = 1
STITCH_FIELDS = ("p", "eps_lo", "eps_hi", "log_err", "n_used", "best")


class FptStitchBin(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in STITCH_FIELDS]


def fpt_stitch(estimates: torch.Tensor, out: Optional[torch.Tensor] = None, *, estimator=ESTIMATOR_LOGNORMAL,
               min_count: int = 400, p_threshold: float = 0.005, stream=None) -> torch.Tensor:
    """Multi-bias reconstruction: estimates float64[n_runs, n_bins, 16] (the
    fpt_estimate outputs of several simulations over the same bins) ->
    float64[n_bins, 6] (STITCH_FIELDS)."""
    if estimates.dim() != 3 or estimates.shape[2] != len(ESTIMATE_FIELDS) or estimates.dtype != torch.float64:
        raise ValueError(f"estimates must be float64[n_runs, n_bins, {len(ESTIMATE_FIELDS)}]")
    n_runs, n_bins = estimates.shape[0], estimates.shape[1]
    if out is None:
        out = torch.empty((n_bins, len(STITCH_FIELDS)), dtype=torch.float64, device=estimates.device)
    _check(lib.fpt_stitch(_dptr(estimates.contiguous()), n_runs, n_bins, estimator, min_count, p_threshold,
                          _dptr(out), _stream(stream)))
    return out


PEARSON_FIELDS = ("r", "count", "mean_N", "mean_lw", "var_N", "var_lw", "cov")


def fpt_pearson(N: torch.Tensor, logw: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> dict:
    """Pearson's r of (N, ln w) over the runs with finite N (device reduction);
    returns {field: float} for PEARSON_FIELDS (synchronises the stream)."""
    if out is None:
        out = torch.empty(8, dtype=torch.float64, device=N.device)
    _check(lib.fpt_pearson(_dptr(N, torch.float64), _dptr(logw, torch.float64), N.numel(), _dptr(out, torch.float64),
                           _stream(stream)))
    v = out.cpu().tolist()
    return {f: v[i] for i, f in enumerate(PEARSON_FIELDS)}


def fpt_normals(seed: int, traj: int, set_id: int, k0: int, n_blocks: int, precision, out: torch.Tensor,
                stream=None):
    prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    _check(lib.fpt_normals(seed, traj, set_id, k0, n_blocks, prec, _dptr(out), _stream(stream)))


MLP_HIDDEN = 64
MLP_NPARAM = 4417
MLP_NPARAM_PAD = 4424
MLP_BYTES = 16 + 2 * MLP_NPARAM_PAD  # sizeof(fpt_mlp_params)


def mlp_pack(params, norm, device="cuda") -> torch.Tensor:
    """fpt_mlp_params as a uint8 device tensor from float parameters (rounded to
    BF16 by round-to-nearest-even) and the 4 input-normalisation constants."""
    p = torch.as_tensor(params, dtype=torch.float32).flatten()
    if p.numel() != MLP_NPARAM:
        raise ValueError(f"expected {MLP_NPARAM} parameters")
    bf = torch.zeros(MLP_NPARAM_PAD, dtype=torch.bfloat16)
    bf[:MLP_NPARAM] = p.to(torch.bfloat16)
    head = torch.as_tensor(norm, dtype=torch.float32).flatten()
    buf = torch.cat([head.view(torch.uint8), bf.view(torch.uint8)])
    assert buf.numel() == MLP_BYTES
    return buf.to(device)


def mlp_unpack_bf16(params) -> torch.Tensor:
    """The float64 values the BF16-rounded parameters represent (what the GPU uses)."""
    p = torch.as_tensor(params, dtype=torch.float32).flatten()
    return p.to(torch.bfloat16).to(torch.float64)


RECORD_FIELDS = 4  # fpt_mlp_record: phi, N, xi_sum (float32), run (uint32)


def fpt_simulate_mlp(params: FptParams, sets: ctypes.Array, seed: int, out_N: torch.Tensor,
                     out_logw: torch.Tensor, records: Optional[torch.Tensor] = None) -> int:
    """Learned-bias simulation; records: float32 device tensor [capacity, 4]
    (column 3 holds the uint32 run index bits).  Returns the number of blocks."""
    n = ctypes.c_int64()
    cap = 0 if records is None else records.shape[0]
    _check(lib.fpt_simulate_mlp(ctypes.byref(params), sets, len(sets), seed, _dptr(out_N, torch.float64),
                                _dptr(out_logw, torch.float64), _dptr(records), cap, ctypes.byref(n)))
    return n.value


class MlpTrainer:
    """Device buffers of fpt_mlp_train_step for one parameter set (allocation
    and the call only; every step runs in the library's kernels)."""

    def __init__(self, spec, params, norm, *, k_eval=32, device="cuda", stream=None):
        self.spec = spec
        self.k_eval = k_eval
        self.norm = tuple(norm)
        n = spec.n_traj
        cap = int(n * (spec.n_max / spec.dN / k_eval + 2))
        f32 = dict(dtype=torch.float32, device=device)
        self.master = torch.as_tensor(params, dtype=torch.float32).to(device).contiguous()
        self.adam_m = torch.zeros(MLP_NPARAM, **f32)
        self.adam_v = torch.zeros(MLP_NPARAM, **f32)
        self.grad = torch.zeros(MLP_NPARAM, **f32)
        self.w = mlp_pack(self.master.cpu(), norm, device)
        self.records = torch.empty((cap, RECORD_FIELDS), **f32)
        self.out_N = torch.empty(n, dtype=torch.float64, device=device)
        self.out_logw = torch.empty(n, dtype=torch.float64, device=device)
        self.coef = torch.empty(n, dtype=torch.float64, device=device)
        self.rows = torch.empty(3 * cap, **f32)
        st = FptMlpTrainState()
        st.master, st.adam_m, st.adam_v = self.master.data_ptr(), self.adam_m.data_ptr(), self.adam_v.data_ptr()
        st.grad, st.w, st.records = self.grad.data_ptr(), self.w.data_ptr(), self.records.data_ptr()
        st.record_capacity = cap
        st.out_N, st.out_logw = self.out_N.data_ptr(), self.out_logw.data_ptr()
        st.coef, st.rows, st.step = self.coef.data_ptr(), self.rows.data_ptr(), 0
        self.state = st
        self.sets = make_sets([spec])
        self.params = make_params(precision=PREC_F32_F64ACC, m=spec.m, n_max=spec.n_max, mlp=self.w,
                                  k_eval=k_eval, stream=stream)

    def step(self, seed: int, tail_N: float, lr: float):
        stats = FptMlpTrainStats()
        _check(lib.fpt_mlp_train_step(ctypes.byref(self.params), self.sets, seed, tail_N, lr,
                                      ctypes.byref(self.state), ctypes.byref(stats)))
        return {"log_second_moment": stats.log_second_moment, "p_hat": stats.p_hat, "n_eff": stats.n_eff,
                "frac_in_tail": stats.frac_in_tail, "n_records": stats.n_records}


def fpt_mlp_forward(w: torch.Tensor, phi: torch.Tensor, N: torch.Tensor, out_b: torch.Tensor, stream=None):
    _check(lib.fpt_mlp_forward(_dptr(w), _dptr(phi, torch.float32), _dptr(N, torch.float32), phi.numel(),
                               _dptr(out_b, torch.float32), _stream(stream)))


def fpt_mlp_backward(w: torch.Tensor, phi: torch.Tensor, N: torch.Tensor, g: torch.Tensor, grad: torch.Tensor,
                     stream=None):
    _check(lib.fpt_mlp_backward(_dptr(w), _dptr(phi, torch.float32), _dptr(N, torch.float32),
                                _dptr(g, torch.float32), phi.numel(), _dptr(grad, torch.float32),
                                _stream(stream)))


def fpt_autotune(params: FptParams, sets: ctypes.Array, seed: int = 0, fraction: float = 0.01):
    """Returns (block_dim, k_steps, pilot steps/s) and caches the shape in the library."""
    b = ctypes.c_int32()
    k = ctypes.c_int32()
    r = ctypes.c_double()
    _check(lib.fpt_autotune(ctypes.byref(params), sets, len(sets), seed, fraction, ctypes.byref(b),
                            ctypes.byref(k), ctypes.byref(r)))
    return b.value, k.value, r.value


def fpt_autotune_reset():
    lib.fpt_autotune_reset()


def fpt_hist_merge(parts, part_counts=None):
    """Histogram of the union of disjoint run sets.  parts: float64 array
    [n_parts, n_bins, BIN_FIELDS] (host; fpt_bin layout, count as int64 bits);
    part_counts: int64 [n_parts, 4] or None.  Returns (bins [n_bins, BIN_FIELDS],
    counts [4] or None) as host tensors."""
    p = torch.as_tensor(parts).detach().to("cpu", torch.float64).contiguous()
    if p.dim() != 3 or p.shape[2] != BIN_FIELDS:
        raise ValueError("parts must be [n_parts, n_bins, BIN_FIELDS]")
    out = torch.empty((p.shape[1], BIN_FIELDS), dtype=torch.float64)
    pc = oc = None
    if part_counts is not None:
        pc = torch.as_tensor(part_counts).detach().to("cpu", torch.int64).contiguous()
        oc = torch.empty(4, dtype=torch.int64)
    _check(lib.fpt_hist_merge(p.data_ptr(), p.shape[0], p.shape[1], None if pc is None else pc.data_ptr(),
                              out.data_ptr(), None if oc is None else oc.data_ptr()))
    return out, oc


def fpt_pipe_rates(stream=None) -> dict:
    """Measured thread operations per second of the FP64 FMA, XU (lg2), wide
    integer multiply and FP32 FMA pipes of the current device."""
    r = FptPipeRates()
    _check(lib.fpt_pipe_rates(ctypes.byref(r), _stream(stream)))
    return {name: getattr(r, name) for name, _ in FptPipeRates._fields_}


def fpt_wait_selftest(stream=None):
    """(expired, seconds) of the library's bounded wait on an mbarrier that
    nothing arrives at (it must expire)."""
    ex = ctypes.c_int32()
    sec = ctypes.c_double()
    _check(lib.fpt_wait_selftest(ctypes.byref(ex), ctypes.byref(sec), _stream(stream)))
    return bool(ex.value), sec.value


# ---- conveniences (allocation + unpacking; no arithmetic of the method) ----

def empty_bins(n_bins: int, device="cuda") -> torch.Tensor:
    return torch.empty((n_bins, BIN_FIELDS), dtype=torch.float64, device=device)


def empty_counts(n: int = 1, device="cuda") -> torch.Tensor:
    return torch.empty((n, 4), dtype=torch.int64, device=device)


def bins_to_numpy(bins: torch.Tensor):
    """(fields float64[n, 7], count int64[n]) from an fpt_bin array."""
    b = bins.detach().cpu().contiguous()
    f = b.numpy()[:, :7].copy()
    c = b.view(torch.int64).numpy()[:, 7].copy()
    return f, c


def empty_estimates(n_bins: int, device="cuda") -> torch.Tensor:
    return torch.empty((n_bins, len(ESTIMATE_FIELDS)), dtype=torch.float64, device=device)


def estimates_to_dict(est: torch.Tensor) -> dict:
    """{field: float64 numpy array [n_bins]} from fpt_estimate's output."""
    a = est.detach().cpu().numpy()
    return {f: a[:, i].copy() for i, f in enumerate(ESTIMATE_FIELDS)}


def lognormal_applies(est: dict, threshold: float = 0.005, min_count: int = 400) -> bool:
    """The rule of §2.4: the lognormal estimate is used when no bin's normality
    p-value falls below the threshold (0.5 %).  The bins tested are those the
    histogram keeps, >= min_count runs (§2.1 truncates bins below 400 runs);
    the test itself needs 8."""
    import numpy as np
    p = est["p_normal"][est["count"] >= min_count]
    p = p[np.isfinite(p)]
    return bool(np.all(p >= threshold))


def simulate_workload(workload, *, block_dim=0, k_steps=0, device="cuda", with_hist=True, stream=None,
                      steps_out=None):
    """Run all sets of a workloads.Workload in one batched call.  Returns
    (N, logw, bins, counts) device tensors."""
    specs = workload.sets
    sets = make_sets(specs)
    n = sum(s.n_traj for s in specs)
    N = torch.empty(n, dtype=torch.float64, device=device)
    lw = torch.empty(n, dtype=torch.float64, device=device)
    bins = counts = None
    if with_hist:
        bins = empty_bins(sum(s.n_bins for s in specs), device)
        counts = empty_counts(len(specs), device)
    s0 = specs[0]
    p = make_params(model=s0.model, precision=workload.precision, m=s0.m, a0=s0.a0, s0=s0.s0,
                    n_max=s0.n_max, block_dim=block_dim, k_steps=k_steps, stream=stream,
                    steps_out=steps_out)
    fpt_simulate_batch(p, sets, workload.seed, N, lw, bins, counts)
    return N, lw, bins, counts
