"""Builds libigr.so, the CUDA library behind include/igr.h, for sm_103a.

The kernel source igr_kernels.cu is compiled once per storage form (FP64,
FP32, FP16, BF16, and FP16/BF16 increments on an FP32 state); the host runtime igr_api.cu and the allocation-free entry
point igr_noalloc.cu once each; the objects compile in parallel and link
into paper_2505_07392_gb300/libigr.so.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libigr.so")
# the bounds-checking debug build (IGR_DEBUG_BOUNDS; include/igr.h)
OBJ_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libigr_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-diag-suppress", "177"]

# (tag, storage type, state type): the increment modes keep the state q^n in
# FP32 and store 16-bit stage increments, Sigma and b
VARIANTS = [("f64", "double", None), ("f32", "float", None), ("f16", "__half", None),
            ("bf16", "__nv_bfloat16", None), ("f16inc", "__half", "float"), ("bf16inc", "__nv_bfloat16", "float")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libigr.so")
    return exe


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".h", ".cuh"))] + \
        [os.path.join(HERE, "..", "include", "igr.h")]


def _jobs(extra, obj):
    jobs = []
    for tag, ty, base in VARIANTS:
        jobs.append([nvcc(), *ARCH, *FLAGS, *extra, f"-DIGR_STORAGE={ty}", f"-DIGR_OPS=ops_{tag}",
                     *([f"-DIGR_BASE={base}"] if base else []),
                     "-c", os.path.join(CSRC, "igr_kernels.cu"), "-o", os.path.join(obj, f"kern_{tag}.o")])
    for name in ("igr_api", "igr_noalloc"):
        jobs.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, name + ".cu"),
                     "-o", os.path.join(obj, name + ".o")])
    return jobs


def build(force: bool = False, verbose: bool = False, extra=(), debug_bounds: bool = False) -> str:
    """Compile and link libigr.so (libigr_debug.so with debug_bounds) if it is
    missing or older than a source."""
    lib, obj = (LIB_DEBUG, OBJ_DEBUG) if debug_bounds else (LIB, OBJ)
    extra = list(extra) + (["-DIGR_DEBUG_BOUNDS"] if debug_bounds else [])
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(f) for f in _sources())
        if os.path.getmtime(lib) >= newest:
            return lib
    os.makedirs(obj, exist_ok=True)
    jobs = _jobs(extra, obj)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        print("\n".join(logs))
    objs = [j[-1] for j in jobs]
    tmp = lib + f".tmp{os.getpid()}"
    run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    xv = ["-Xptxas", "-v"] if "-v" in sys.argv else []
    print(build(force=True, verbose=bool(xv), extra=xv))
