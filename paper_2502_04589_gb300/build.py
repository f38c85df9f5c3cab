"""Build libpase.so in-tree for sm_103a (nvcc + g++, translation units compiled in parallel)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpase.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["sparse_kernels.cu", "dense_kernels.cu", "pase.cu", "noalloc.cu", "smoother.cu", "split_gemm.cu", "stencil.cu", "df64.cu", "flow.cu"]
CPP = ["host_setup.cpp"]


def _nvcc():
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def sources():
    return [os.path.join(CSRC, f) for f in CU + CPP] + [
        os.path.join(CSRC, "pase_internal.h"), os.path.join(CSRC, "tc_util.h"),
        os.path.join(HERE, "..", "include", "pase.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(verbose=False, force=False, ptxas_info=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
               "-c", os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for f in CPP:
        obj = os.path.join(BUILD, f + ".o")
        inc = os.path.join(os.path.dirname(nvcc), "..", "include")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-I" + inc, "-c",
               os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-Xcompiler", "-fopenmp",
          "-lgomp", "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
