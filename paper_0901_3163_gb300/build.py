"""Build the dlz CUDA library in-tree: paper_0901_3163_gb300/libdlz.so (sm_103a).

    python -m paper_0901_3163_gb300.build        (or build() from Python)

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library against the shared CUDA runtime.  Objects go to
paper_0901_3163_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdlz.so")
SOURCES = ["wilson.cu", "wilson_eo.cu", "wilson_bf16.cu", "dr.cu", "solvers.cu", "solvers_mixed.cu", "minres_fused.cu",
           "cg_fused.cu", "minres_multi.cu", "gmres.cu", "api.cu", "ptc.cu", "tc_gemm.cu", "small_dense.cpp", "small_dense_z.cpp", "restart_plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags(debug=False):
    f = ["-std=c++17", "-O3", "-lineinfo", "--extended-lambda", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fno-strict-aliasing", "-I", os.path.join(HERE, "..", "include")]
    if debug:
        f += ["-DDLZ_DEBUG"]
    return f + ARCH


def _newest_input():
    paths = [os.path.join(CSRC, p) for p in os.listdir(CSRC)]
    paths.append(os.path.join(HERE, "..", "include", "dlz.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libdlz.so if any source is newer than it; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags()
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj] + _flags()
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared",
                                                         "-Xlinker", "-rpath=/usr/local/cuda/lib64",
                                                         "-Xlinker", "--no-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
