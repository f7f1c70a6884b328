"""Build libmarnoldi (CUDA for sm_103a) in-tree with nvcc.

The translation units compile in parallel to object files, then nvcc links
them into ``_build/libmarnoldi_<machine>.so``.  Nothing is installed outside
the package directory.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "krylov.cu", "eigsub.cu", "outputs.cu", "region.cu", "support.cu", "noalloc.cu",
           "server.cu", "eigstate.cu", "gs_stream.cu"]
HEADERS = [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "gs_common.cuh"), os.path.join(INCLUDE, "marnoldi.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmarnoldi")


def lib_path(variant: str = "") -> str:
    """The library of the default build, or of a variant ("check": built with
    -DMARNOLDI_CHECK, index checks in the kernels)."""
    tag = f"_{variant}" if variant else ""
    return os.path.join(BUILD, f"libmarnoldi{tag}_{platform.machine()}.so")


VARIANTS = {"": [], "check": ["-DMARNOLDI_CHECK"]}


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          variant: str = "") -> str:
    """Compile (if stale) and link libmarnoldi (or a variant of it, see VARIANTS); returns the
    library path."""
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + VARIANTS[variant] + list(extra_flags or [])
    mach = platform.machine() + (f"_{variant}" if variant else "")
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, f"{os.path.splitext(src)[0]}_{mach}.o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([cc, *ARCH, *flags, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose and (r.stdout or r.stderr):
                    print(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(j)}\n{r.stdout}{r.stderr}")
    out = lib_path(variant)
    if force or jobs or _stale(out, objs):
        tmp = out + f".tmp{os.getpid()}"
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}{r.stderr}")
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
