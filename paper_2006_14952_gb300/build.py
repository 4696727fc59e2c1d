"""Compile libhfmm.so for sm_103a (in-tree, no cmake).

Each ``csrc/*.cu`` is compiled by its own nvcc process in parallel, then linked
with ``nvcc -shared``.  The result lands in ``paper_2006_14952_gb300/_build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhfmm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


GENERATED = os.path.join(CSRC, "gen_bodies.cuh")


def _generate():
    """Straight-line expansion bodies (gen_bodies.py); rewritten only when they change."""
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_bodies.py"), GENERATED])


def _inputs():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) +
            [os.path.join(CSRC, "gen_bodies.py")])


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(GENERATED):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _inputs())


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def _stale(src: str, headers_mtime: float) -> bool:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    return not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), headers_mtime)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the stale objects (source or any shared header newer than the object) and link."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and up_to_date():
        return LIB
    _generate()
    srcs = sources()
    hdr = max(os.path.getmtime(h) for h in _inputs() if not h.endswith(".cu"))
    todo = srcs if force else [s for s in srcs if _stale(s, hdr)]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcufft", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
