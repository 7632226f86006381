"""Build the JFNK CUDA library (libjfnk.so) in-tree for sm_103a with nvcc.

Usage: python -m paper_1512_03662_gb300.build  (or build() from Python).
The translation units compile in parallel; the shared library lands in
paper_1512_03662_gb300/_build/.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libjfnk.so")
SOURCES = ["residual.cu", "krylov.cu", "precond.cu", "adjoint.cu", "engine.cu", "noalloc.cu"]
# the FP64 throughput probe of the benchmark: a library of its own, not part of the solver's C ABI
PROBE_SOURCE = "fp64_probe.cu"
PROBE_LIB = os.path.join(BUILD, "libfp64probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                   "-I", CSRC] + list(extra)


def _newer(target, deps):
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "jfnk.h"))
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not _newer(o, [s] + headers):
            jobs.append([cc, "-c", s, "-o", o] + _flags(extra))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {cmd[2]}")
        return r

    ps = os.path.join(CSRC, PROBE_SOURCE)
    if force or not _newer(PROBE_LIB, [ps] + headers):
        jobs.append([cc, "-shared", ps, "-o", PROBE_LIB] + _flags(extra) + ["-lcudart"])
    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if any(j[2] != ps for j in jobs) or not os.path.exists(LIB):
        run([cc, "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
