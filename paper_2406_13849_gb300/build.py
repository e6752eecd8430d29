"""Build the C-ABI library in-tree (no cmake, one -gencode, parallel compiles).

Produces, under ``paper_2406_13849_gb300/_build/``:
  libtrk.so        fast build (FP64 contraction allowed)
  libtrk_exact.so  --fmad=false build, bit-exact against the FP64 oracle
Both link the same host object (geometry_build.cpp, -ffp-contract=off).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# translation units compiled once per flavour (fast / exact)
KERNEL_UNITS = ["trk_kernels", "trk_event", "batch"]
# translation units compiled once and linked into both flavours
SHARED_UNITS = ["peaks", "noalloc"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".h"))] + [os.path.join(INCLUDE, "trk.h")]


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in _sources())


def outputs():
    return {"fast": os.path.join(BUILD, "libtrk.so"), "exact": os.path.join(BUILD, "libtrk_exact.so")}


def build(force: bool = False, verbose: bool = False) -> dict:
    """Compile (if stale) and return the paths of both libraries.

    TRK_NVCC_FLAGS (environment) adds flags to the kernel compiles, e.g.
    -DTRK_EV_MINB=2 to change a kernel's register budget."""
    outs = outputs()
    if not force and not any(_stale(p) for p in outs.values()):
        return outs
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    host_obj = os.path.join(BUILD, "geometry_build.o")
    jobs = [
        ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-Wall"] + inc +
        ["-I" + os.path.join(cuda, "include"), "-c", os.path.join(CSRC, "geometry_build.cpp"), "-o", host_obj],
    ]
    shared_objs = []
    for unit in SHARED_UNITS:
        obj = os.path.join(BUILD, unit + ".o")
        shared_objs.append(obj)
        jobs.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"] + inc +
                    ["-c", os.path.join(CSRC, unit + ".cu"), "-o", obj])
    extra_flags = os.environ.get("TRK_NVCC_FLAGS", "").split()
    kobjs = {"fast": [], "exact": []}
    for flavour, extra in (("fast", []), ("exact", ["--fmad=false", "-DTRK_EXACT"])):
        for unit in KERNEL_UNITS:
            obj = os.path.join(BUILD, f"{unit}_{flavour}.o")
            kobjs[flavour].append(obj)
            jobs.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                         "-Xcompiler", "-ffp-contract=off"] + extra + extra_flags + inc +
                        ["-c", os.path.join(CSRC, unit + ".cu"), "-o", obj])
    procs = [subprocess.Popen(j, stdout=None if verbose else subprocess.PIPE,
                              stderr=subprocess.STDOUT) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((j, out.decode() if out else ""))
    if failed:
        msg = "\n".join(" ".join(j) + "\n" + o for j, o in failed)
        raise RuntimeError("library build failed:\n" + msg)
    for flavour, target in outs.items():
        tmp = target + ".tmp"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp, host_obj] + kobjs[flavour] + shared_objs +
                       ["-lcudart"], check=True)
        os.replace(tmp, target)
    return outs


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
