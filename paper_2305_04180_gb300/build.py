"""Build the CUDA library ``libsparrowgb.so`` in-tree for sm_103a.

Every translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) and linked against the shared
CUDA runtime, so that the library and PyTorch share one runtime instance.
The simulator translation units use ``-fmad=false``: the step is defined as
an exact float32 expression tree and fused multiply-adds appear only where
the code writes fmaf().
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsparrowgb.so")
# the debug variant: explicit bounds checks that latch SG_DEV_BOUNDS instead
# of reading outside an array (see sg_sim_status in the header)
DEBUG_LIB = os.path.join(BUILD, "debug", "libsparrowgb_debug.so")
VARIANTS = {"": (LIB, []), "debug": (DEBUG_LIB, ["-DSG_DEBUG_BOUNDS"])}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# per-file extra flags
UNITS = {
    "sg_sim.cu": ["-fmad=false"],
    "sg_qnet.cu": ["-fmad=false"],
    "sg_graph.cu": [],
    "sg_probe.cu": [],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsparrowgb.so")


def _sources():
    return [os.path.join(CSRC, f) for f in UNITS]


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "sparrow_gb.h"))
    out.append(__file__)
    return out


def up_to_date(variant: str = "") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=None, variant: str = "") -> str:
    """Compile and link the library (variant "" or "debug"); returns its path."""
    lib, vflags = VARIANTS[variant]
    if not force and up_to_date(variant):
        return lib
    out_dir = os.path.dirname(lib)
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    extra = list(vflags) + list(extra or [])

    def compile_one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(out_dir, name.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *UNITS[name], *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                variant="debug" if "--debug" in sys.argv else ""))
