"""The C-ABI library loads on a machine without a GPU, exports every function
declared in include/fpt.h, and rejects invalid arguments on the host before
touching the GPU (no compute calls here)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fpt.h")


@pytest.fixture(scope="module")
def native():
    from paper_2206_11234_gb300 import build
    build.build()
    from paper_2206_11234_gb300 import native
    return native


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fpt_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported(native):
    names = declared_functions()
    assert "fpt_simulate" in names and "fpt_histogram" in names and len(names) >= 7
    for name in names:
        assert hasattr(native.lib, name), name


def test_struct_layouts_match_header(native, tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives
    the header's structs."""
    structs = {"fpt_params": native.FptParams, "fpt_set": native.FptSet, "fpt_bin": native.FptBin,
               "fpt_hist_counts": native.FptHistCounts, "fpt_mlp_train_state": native.FptMlpTrainState,
               "fpt_mlp_train_stats": native.FptMlpTrainStats, "fpt_estimate_bin": native.FptEstimateBin,
               "fpt_stitch_bin": native.FptStitchBin, "fpt_pipe_rates_out": native.FptPipeRates}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fpt.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('printf("fpt_mlp_params %zu\\n", sizeof(fpt_mlp_params));')
    lines.append('printf("fpt_mlp_record %zu\\n", sizeof(fpt_mlp_record));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["cc", "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["fpt_mlp_params"]) == native.MLP_BYTES
    assert int(out["fpt_mlp_record"]) == 4 * native.RECORD_FIELDS
    for cname, cls in structs.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def _params(native, **kw):
    p = native.FptParams()
    p.abi_version = native.FPT_ABI_VERSION
    p.model = native.MODEL_QUADRATIC
    p.precision = native.PREC_F64
    p.bias_kind = native.BIAS_CONST
    p.m = 1.0
    p.n_max = 6.0
    p.stream = None
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_host_side_argument_checks(native):
    L = native.lib
    buf = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its checks first
    sq2 = math.sqrt(2.0)

    def sim(p, n=8, phi_in=3.0, phi_end=sq2, phi_uv=math.inf, dN=1e-3, b=1.0, out=buf):
        return L.fpt_simulate(ctypes.byref(p) if p is not None else None, n, phi_in, phi_end, phi_uv,
                              dN, b, 0, out, out)

    E = native.FPT_EINVAL
    assert sim(None) == E
    assert sim(_params(native, abi_version=99)) == E
    assert sim(_params(native, model=7)) == E
    assert sim(_params(native, precision=9)) == E
    assert sim(_params(native, bias_kind=5)) == E
    assert sim(_params(native, bias_kind=native.BIAS_MLP)) == native.FPT_EUNSUPPORTED
    assert sim(_params(native, block_dim=100)) == E
    assert sim(_params(native, block_dim=1024)) == E
    assert sim(_params(native, model=native.MODEL_CONSTANT, s0=0.0)) == E
    assert sim(_params(native), n=-1) == E
    assert sim(_params(native), out=None) == E
    assert sim(_params(native), dN=0.0) == E
    assert sim(_params(native), dN=-1.0) == E
    assert sim(_params(native), dN=math.nan) == E
    assert sim(_params(native), phi_uv=2.0) == E
    assert sim(_params(native), phi_uv=math.nan) == E
    assert sim(_params(native), phi_in=math.inf) == E
    assert sim(_params(native), b=math.inf) == E
    assert sim(_params(native, n_max=math.inf)) == E
    assert sim(_params(native, n_max=0.0)) == E
    assert sim(_params(native, n_max=1e9)) == E  # beyond 2^31 steps
    assert sim(_params(native, m=0.0)) == E
    # polynomial potential: zero, non-finite, or non-positive where runs start
    assert sim(_params(native, model=native.MODEL_POLYNOMIAL)) == E
    pp = _params(native, model=native.MODEL_POLYNOMIAL)
    pp.poly[2] = math.nan
    assert sim(pp) == E
    pp.poly[2] = -1.0
    assert sim(pp) == E
    assert b"dN" in L.fpt_last_error() or len(L.fpt_last_error()) > 0
    # n_traj = 0 is a no-op that needs no GPU
    assert sim(_params(native), n=0, out=None) == native.FPT_OK
    # histogram
    h = lambda n, nb, lo, hi, ns: L.fpt_histogram(buf, buf, n, nb, lo, hi, ns, 0, buf, buf, None)
    assert h(-1, 8, 0.0, 1.0, 1) == E
    assert h(8, 0, 0.0, 1.0, 1) == E
    assert h(8, 8, 1.0, 1.0, 1) == E
    assert h(8, 8, 0.0, math.inf, 1) == E
    assert h(8, 4097, 0.0, 1.0, 1) == E
    assert h(8, 1024, 0.0, 1.0, 5) == E
    assert h(8, 8, 0.0, 1.0, 0) == E
    assert L.fpt_histogram(None, buf, 8, 8, 0.0, 1.0, 1, 0, buf, buf, None) == E
    # estimates of a histogram
    est = lambda nb, ns, lo, hi, n: L.fpt_estimate(buf, nb, ns, lo, hi, n, 0, buf, None)
    assert est(0, 1, 0.0, 1.0, 10) == E
    assert est(8, 0, 0.0, 1.0, 10) == E
    assert est(1024, 5, 0.0, 1.0, 10) == E
    assert est(8, 1, 1.0, 0.0, 10) == E
    assert est(8, 1, 0.0, math.nan, 10) == E
    assert est(8, 1, 0.0, 1.0, 0) == E
    assert L.fpt_estimate(None, 8, 1, 0.0, 1.0, 10, 0, buf, None) == E
    st = lambda nr, nb, est_kind, mc, pt: L.fpt_stitch(buf, nr, nb, est_kind, mc, pt, buf, None)
    assert st(0, 8, 1, 400, 0.005) == E
    assert st(2, 0, 1, 400, 0.005) == E
    assert st(2, 8, 7, 400, 0.005) == E
    assert st(2, 8, 1, 1, 0.005) == E
    assert st(2, 8, 1, 400, 1.0) == E
    assert st(2, 8, 1, 400, math.nan) == E
    assert L.fpt_stitch(None, 2, 8, 1, 400, 0.0, buf, None) == E
    # batch
    sets = (native.FptSet * 2)()
    for s in sets:
        s.phi_in, s.phi_end, s.phi_uv, s.m, s.b, s.dN, s.n_max, s.n_traj = 3.0, sq2, math.inf, 1.0, 1.0, 1e-3, 6.0, 4
        s.n_bins, s.hist_lo, s.hist_hi = 10, 0.0, 6.0
    p = _params(native)
    assert L.fpt_simulate_batch(ctypes.byref(p), sets, 0, 0, buf, buf, None, None) == E
    assert L.fpt_simulate_batch(ctypes.byref(p), sets, 65, 0, buf, buf, None, None) == E
    assert L.fpt_simulate_batch(ctypes.byref(p), None, 1, 0, buf, buf, None, None) == E
    assert L.fpt_simulate_batch(ctypes.byref(p), sets, 2, 0, buf, buf, buf, None) == E
    sets[1].n_bins = 0
    assert L.fpt_simulate_batch(ctypes.byref(p), sets, 2, 0, buf, buf, buf, buf) == E
    assert L.fpt_simulate_batch_host(ctypes.byref(p), sets, 2, 0, None, None, None, None) == E
    assert L.fpt_normals(0, 0, 0, 0, -1, 0, buf, None) == E
    assert L.fpt_normals(0, 0, 0, 0xFFFFFFFF, 2, 0, buf, None) == E


def test_strerror_names_every_code(native):
    L = native.lib
    for code in (0, -1, -2, -3, -4, -5):
        assert L.fpt_strerror(code) != b"unknown error"
    assert L.fpt_strerror(-99) == b"unknown error"
    assert L.fpt_abi_version() == native.FPT_ABI_VERSION


def test_injection_entries_validate_on_the_host(native):
    L = native.lib
    assert L.fpt_inject_alloc_failures(-1) == native.FPT_EINVAL
    assert L.fpt_inject_alloc_failures(0) == native.FPT_OK
    assert L.fpt_inject_status(0) == native.FPT_OK
