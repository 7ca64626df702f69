"""Build libgrb.so (the CUDA library behind include/grb.h) in-tree.

Every translation unit under csrc/ is compiled by nvcc for sm_103a only, in
parallel, and linked into paper_2509_14211_gb300/libgrb.so against the shared
CUDA runtime.  The same sources compiled with -DGRB_CHECK_BOUNDS make the
bounds-checked debug library libgrb_checked.so (include/grb_debug.h); both
variants' objects are compiled in one parallel pool.  Objects go to
paper_2509_14211_gb300/_build/ (release) and _build/checked/ and are rebuilt
when a source or any header is newer.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgrb.so")
LIB_CHECKED = os.path.join(PKG, "libgrb_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and not shutil.which(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


VARIANTS = (("", LIB, BUILD), ("-DGRB_CHECK_BOUNDS", LIB_CHECKED, os.path.join(BUILD, "checked")))


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Build libgrb.so (and, unless checked=False, libgrb_checked.so);
    returns the release library's path."""
    nvcc = _nvcc()
    headers = _headers()
    jobs = []
    links = []
    # GRB_NVCC_FLAGS: extra -D tuning knobs (e.g. -DPR_MINBLOCKS=4)
    extra = os.environ.get("GRB_NVCC_FLAGS", "").split()
    for define, lib, bdir in VARIANTS if checked else VARIANTS[:1]:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        nj = len(jobs)
        for src in _sources():
            obj = os.path.join(bdir, os.path.basename(src) + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
                       *([define] if define else []), "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj + ".tmp"]
                jobs.append((cmd, obj))
        links.append((lib, objs, len(jobs) > nj))

    def run(job):
        cmd, obj = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.relpath(obj, PKG)}:\n{r.stderr[-4000:]}")
        os.replace(obj + ".tmp", obj)
        if verbose:
            print("built", os.path.relpath(obj, PKG))

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    for lib, objs, rebuilt in links:
        if force or rebuilt or _stale(lib, objs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
