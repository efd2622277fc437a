"""Build liblqcd.so (the C-ABI CUDA library) in-tree for sm_103a.

Each csrc/*.cu is compiled by nvcc in parallel, then linked into
paper_1112_5280_gb300/_build/liblqcd.so. A rebuild happens only when a
source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblqcd.so")
# the debug build: device bounds checks on every field access (LQCD_DEBUG_BOUNDS)
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "liblqcd.so")


def lib_path(debug: bool = False) -> str:
    return LIB_DEBUG if debug else LIB

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"] + ARCH


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(debug: bool = False) -> bool:
    lib = lib_path(debug)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src, extra, outdir=BUILD):
    obj = os.path.join(outdir, os.path.basename(src)[:-3] + ".o")
    # LQCD_NVCC_EXTRA: extra nvcc flags, e.g. -D values of the compile-time tunables
    env_extra = os.environ.get("LQCD_NVCC_EXTRA", "").split()
    cmd = [_nvcc()] + NVCC_FLAGS + extra + env_extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, debug: bool = False) -> str:
    """Compile and link the library (debug=True: the bounds-checked build, in its own folder)."""
    lib = lib_path(debug)
    outdir = os.path.dirname(lib)
    if not force and up_to_date(debug):
        return lib
    os.makedirs(outdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    if debug:
        extra = extra + ["-DLQCD_DEBUG_BOUNDS"]
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, outdir), srcs))
    if verbose or ptxas_verbose:
        for _, err in results:
            if err:
                print(err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv))


# Files that define the Dslash kernel and its launch (a change to any of them
# invalidates profile counters taken on the old code).
DSLASH_KERNEL_FILES = ("field.cuh", "dslash.cuh", "batch.cuh", "kernels.cuh", "kernels_inst.cuh",
                       "kernels_f32.cu", "kernels_f16.cu", "kernels_f64.cu", "launch.h", "layout.cu")


def source_hash(files=DSLASH_KERNEL_FILES) -> str:
    """Hash of the kernel sources' code (ties profile counters to the code they were taken
    on). Comments and blank lines are left out, so that editing a comment keeps the
    counters; any change to the code itself changes the hash."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in sorted(files):
        txt = open(os.path.join(CSRC, name)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        txt = "\n".join(line.rstrip() for line in txt.split("\n") if line.strip())
        h.update(name.encode())
        h.update(txt.encode())
    return h.hexdigest()[:16]
