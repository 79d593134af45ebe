"""Build libbitssa.so in-tree with nvcc for sm_103a.

The bit-sliced kernel is instantiated once per number of propensity planes K
(1..31); each instantiation is its own object file built from
``csrc/frank_instance.cu`` with ``-DBITSSA_K=<K>`` so that they compile in
parallel.  Objects go to ``_build/`` next to this file; the library is
``libbitssa.so`` in the package directory.  The lattice kernel is instantiated once
per count-plane width (4, 8, 12, 16) from ``csrc/lattice_instance.cu``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbitssa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
K_VALUES = list(range(1, 32))
LATTICE_PLANES = (4, 8, 12, 16)  # count planes of the lattice kernel's instantiations


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libbitssa")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "-I", INCLUDE, "-I", CSRC]


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _jobs():
    jobs = []
    for k in K_VALUES:
        jobs.append((os.path.join(CSRC, "frank_instance.cu"), os.path.join(BUILD, f"frank_k{k:02d}.o"),
                     [f"-DBITSSA_K={k}"]))
        jobs.append((os.path.join(CSRC, "frank_trio_instance.cu"), os.path.join(BUILD, f"frank_trio_k{k:02d}.o"),
                     [f"-DBITSSA_K={k}"]))
        jobs.append((os.path.join(CSRC, "general_instance.cu"), os.path.join(BUILD, f"general_k{k:02d}.o"),
                     [f"-DBITSSA_K={k}"]))
    for p in LATTICE_PLANES:
        jobs.append((os.path.join(CSRC, "lattice_instance.cu"), os.path.join(BUILD, f"lattice_p{p:02d}.o"),
                     [f"-DBITSSA_LAT_P={p}"]))
    for name in ("frank_dispatch", "thread_per_run", "runtime", "selftest", "noalloc", "lattice"):
        jobs.append((os.path.join(CSRC, name + ".cu"), os.path.join(BUILD, name + ".o"), []))
    return jobs


def _stale(out, src, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in [src] + deps)


def build(force: bool = False, verbose: bool = False, workers: int | None = None) -> str:
    """Compile every translation unit that is out of date and link libbitssa.so."""
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    deps = _deps()
    todo = [j for j in _jobs() if force or _stale(j[1], j[0], deps)]

    def compile_one(job):
        src, out, extra = job
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc] + _flags() + extra + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(out)}:\n{r.stderr[-4000:]}")
        os.replace(tmp, out)
        if verbose:
            print("built", os.path.basename(out), flush=True)

    if todo:
        with cf.ThreadPoolExecutor(max_workers=workers or os.cpu_count() or 4) as ex:
            for f in [ex.submit(compile_one, j) for j in todo]:
                f.result()
    objs = [j[1] for j in _jobs()]
    if force or todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libbitssa.so failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    import time
    t0 = time.time()
    print(build(force="--force" in sys.argv, verbose=True), f"{time.time() - t0:.1f}s")
