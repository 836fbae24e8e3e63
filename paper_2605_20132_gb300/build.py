"""Build libfilark.so in-tree (paper_2605_20132_gb300/_build/) with nvcc for sm_103a.

The CUDA translation unit and the host C++ units are compiled in parallel and
linked into one shared library with the CUDA runtime linked statically, so the
library does not depend on the runtime that PyTorch ships.  Host code is built
without floating-point contraction and without target-specific flags, so the
planner gives the same tables on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfilark.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["chain_kernel.cu", "chain_kernel_trig.cu", "chain_batch.cu", "chain_batch_solo.cu", "chain_static.cu", "sos_adjoint.cu", "trigger.cu",
              "temporal.cu", "fftfilt.cu", "view.cu"]
CPP_SOURCES = ["plan.cpp", "api.cpp", "batch.cpp"]
HEADERS = [os.path.join(CSRC, "filark_internal.h"), os.path.join(CSRC, "chain_body.cuh"), os.path.join(CSRC, "chain_object.h"),
           os.path.join(CSRC, "chain_batch.cuh"),
           os.path.join(CSRC, "host_trace.h"),
           os.path.join(INCLUDE, "filark.h")]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or CUDA_HOME)")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(nvcc: str, src: str, obj: str, extra: list[str]) -> None:
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE,
           "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", *extra,
           "-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libfilark.so."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = nvcc_path()
    jobs = []
    objs = []
    for name in CU_SOURCES + CPP_SOURCES:
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT, name + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *HEADERS]):
            extra = ["-Xptxas", "-v"] if (verbose and name.endswith(".cu")) else []
            if name.endswith(".cpp"):
                extra = ["-x", "c++"]
            jobs.append((src, obj, extra))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(_compile, nvcc, s, o, e) for s, o, e in jobs]
            for f in futs:
                f.result()
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", LIB + ".tmp", *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
