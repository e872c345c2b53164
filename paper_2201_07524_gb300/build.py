"""Build the sk CUDA library in-tree: one nvcc job per translation unit (run in
parallel), then a shared-library link.  Output: paper_2201_07524_gb300/_build/libsk.so.

Only sm_103a code is generated.  The CUDA runtime is linked statically, so the
library loads (and reports its exports) on machines without a GPU.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsk.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["sk_api.cu", "sk_plan_kernels.cu", "sk_spread.cu", "sk_spread3.cu", "sk_fft.cu", "sk_direct.cu", "sk_nearfield.cu", "sk_noalloc.cu", "sk_tc.cu", "sk_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False, extra_flags=()):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "sk.h"))
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or _newer(LIB, objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    build_example()
    return LIB


EXAMPLE_SRC = os.path.join(HERE, "examples", "sk_example.c")
EXAMPLE = os.path.join(OUT, "sk_example")


def build_example():
    """The plain-C example of the ABI (host compiler, linked against the
    library, found next to it at run time)."""
    if not _newer(EXAMPLE, [EXAMPLE_SRC, LIB, os.path.join(INCLUDE, "sk.h")]):
        return EXAMPLE
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the example")
    cmd = [cc, "-O2", "-std=c11", "-Wall", "-I", INCLUDE, EXAMPLE_SRC, "-L", OUT, "-lsk", "-Wl,-rpath,$ORIGIN",
           "-o", EXAMPLE]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("example build failed")
    return EXAMPLE


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
