"""Build step of libepsr: compiles the CUDA sources for sm_103a into an in-tree shared
library (paper_1904_08756_gb300/libepsr.so). Translation units compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libepsr.so")
# measurements of the GPU for the benchmark, kept out of the product library
PROBE_LIB = os.path.join(HERE, "libepsr_probe.so")
PROBE_SOURCES = ["k_micro.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
SOURCES = ["epsr_api.cu", "k_mc.cu", "k_gr.cu", "k_sq.cu", "k_sq_tc.cu", "k_ep.cu", "k_smear.cu", "epsr_noalloc.cu", "epsr_tune.cu", "epsr_refine.cu"]
# The Monte Carlo kernel's FP32 energies never come near the denormal range (|r| >= grid
# spacing, r <= box diagonal), so denormal support is dropped there (single-instruction rsqrt).
PER_FILE_FLAGS = {"k_mc.cu": ["-ftz=true"]}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libepsr")


def _stale(target: str, deps: list) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "epsr.h"))
    flags = NVCC_FLAGS + (extra_flags or [])
    headers.append(os.path.join(INCLUDE, "epsr_probe.h"))
    objs, probe_objs = [], []
    jobs = []
    for src in SOURCES + PROBE_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        (probe_objs if src in PROBE_SOURCES else objs).append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *flags, *PER_FILE_FLAGS.get(src, []), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-Xlinker", "-soname=libepsr.so", "-lcudart_static",
             "-lrt", "-ldl", "-lpthread"])
        os.replace(tmp, LIB)
    if force or jobs or _stale(PROBE_LIB, probe_objs + [LIB]):
        tmp = PROBE_LIB + f".{os.getpid()}.tmp"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *probe_objs, "-L" + HERE, "-lepsr", "-Xlinker", "-rpath=$ORIGIN",
             "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
        os.replace(tmp, PROBE_LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
