"""Build libfpt_gb300.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2206_11234_gb300/libfpt_gb300.so.  The binary64 stepper and the RNG
probe are compiled with FMA contraction off so that their arithmetic is
rounded exactly as written in the source.

build(debug=True) builds the same sources with -DFPT_DEBUG=1 into
libfpt_gb300_debug.so: kernels whose bounds checks (parameter set of a
ticket, replay-queue capacity, record index, histogram bin index) record a
status bit and skip the access, reported by the call as FPT_EDEVICE_STATUS.
The binding loads it instead of the default library when the environment
variable FPT_DEBUG_LIB is 1.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfpt_gb300.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
UNITS = {
    "abi.cu": [],
    "histogram.cu": [],
    "stepper_f32.cu": [],
    "stepper_pow.cu": [],
    "stepper_f64.cu": ["-fmad=false", "-DFPT_STEPPER_MAXNREG=128"],
    "rng_probe.cu": ["-fmad=false"],
    "noalloc.cu": [],
    "autotune.cu": [],
    "mlp.cu": [],
    "stepper_mlp.cu": [],
    "train.cu": [],
    "plan.cu": [],
    "estimate.cu": [],
    "pipes.cu": [],
    "hist_merge.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fpt.h"))
    files.append(os.path.abspath(__file__))
    return files


LIB_DEBUG = os.path.join(HERE, "libfpt_gb300_debug.so")


def lib_path(debug: bool = False) -> str:
    return LIB_DEBUG if debug else LIB


def up_to_date(debug: bool = False) -> bool:
    lib = lib_path(debug)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = lib_path(debug)
    if not force and up_to_date(debug):
        return lib
    build_dir = BUILD + ("_debug" if debug else "")
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-DFPT_DEBUG=1"] if debug else []

    def compile_unit(name):
        obj = os.path.join(build_dir, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *extra, *UNITS[name], "-c", os.path.join(CSRC, name), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, sorted(UNITS)))
    if verbose:
        for obj, log in results:
            print(obj, log, file=sys.stderr)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
