"""Build libdiaq_gb300.so in-tree (paper_2405_01250_gb300/_build/).

Every CUDA translation unit is compiled for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), in parallel; the host C++ is
compiled with g++; the objects are linked into one shared library against
the shared CUDA runtime (so it joins the runtime PyTorch already loaded).
No cmake, no architecture-specific host flags: the same command builds on
x86 and on Arm hosts.
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdiaq_gb300.so")
# the debug build: every kernel checks its computed indices (-DDIAQ_DEBUG_BOUNDS)
DBG_DIR = os.path.join(HERE, "_build_dbg")
DBG_LIB = os.path.join(DBG_DIR, "libdiaq_gb300_dbg.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, cpp, hdr


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    cu, cpp, hdr = _sources()
    return any(os.path.getmtime(p) > t for p in cu + cpp + hdr + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug_bounds: bool = None) -> str:
    """Build the library (or, with debug_bounds, its index-checking debug
    build; default: the one DIAQ_DEBUG_BOUNDS=1 selects)."""
    if debug_bounds is None:
        debug_bounds = os.environ.get("DIAQ_DEBUG_BOUNDS", "0") == "1"
    out_dir, lib = (DBG_DIR, DBG_LIB) if debug_bounds else (OUT_DIR, LIB)
    if not force and not _stale(lib):
        return lib
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(out_dir, exist_ok=True)
    cu, cpp, _ = _sources()
    common = ["-O3", "-std=c++17", f"-I{INCLUDE}", f"-I{CSRC}"] + (["-DDIAQ_DEBUG_BOUNDS"] if debug_bounds else [])
    jobs = []
    objs = []
    for src in cu:
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, "-gencode", GENCODE, "-lineinfo", "-Xcompiler", "-fPIC", "-c", src, "-o", obj] + common
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append(cmd)
        objs.append(obj)
    for src in cpp:
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = ["g++", "-fPIC", "-Wall", "-c", src, "-o", obj, f"-I{os.path.join(cuda, 'include')}"] + common
        jobs.append(cmd)
        objs.append(obj)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(run, jobs))
    for cmd, p in results:
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        if (verbose or ptxas_info) and (p.stdout or p.stderr):
            print(p.stdout + p.stderr, flush=True)
    tmp = lib + f".{os.getpid()}.tmp"
    link = [nvcc, "-shared", "-cudart", "shared", "-gencode", GENCODE, "-o", tmp] + objs + [
        "-Xlinker", "-rpath", "-Xlinker", os.path.join(cuda, "lib64"),
        "-Xlinker", "-rpath", "-Xlinker", os.path.join(cuda, "lib"),
    ]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv,
                debug_bounds=True if "--debug-bounds" in sys.argv else None))
