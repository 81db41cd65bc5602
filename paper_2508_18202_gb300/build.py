"""Build libsclbm.so in-tree (paper_2508_18202_gb300/_build/) for sm_103a.

nvcc compiles the CUDA translation units for compute_103a/sm_103a only; g++
compiles the host numerics with floating-point contraction disabled so that
quadrature nodes and weights are reproducible bit for bit.  The units are
compiled in parallel and linked into one shared library with static cudart.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsclbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CUDA_UNITS = ["lbm_kernels.cu", "lbm_kernels_rr.cu", "observables.cu", "adjoint.cu", "api.cu", "noalloc.cu",
              "quantiles.cu"]
HOST_UNITS = ["host_numerics.cpp"]
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    srcs = [os.path.join(CSRC, f) for f in CUDA_UNITS + HOST_UNITS]
    srcs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(INCLUDE, "sclbm.h"))
    return srcs


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in _sources()):
            return LIB
    nvcc = _nvcc()
    objs, procs = [], []
    for unit in CUDA_UNITS:
        obj = os.path.join(OUT_DIR, unit + ".o")
        cmd = [nvcc, GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-c", os.path.join(CSRC, unit), "-o", obj] + list(extra_nvcc)
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for unit in HOST_UNITS:
        obj = os.path.join(OUT_DIR, unit + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
               "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, unit), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(" ".join(cmd) + "\n" + text)
        elif verbose and text.strip():
            print(text)
    if failed:
        raise RuntimeError("libsclbm build failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc, GENCODE, "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-lpthread", "-ldl"]
    subprocess.run(link, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
