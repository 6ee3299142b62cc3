"""Build libawe.so (the CUDA library behind include/awe.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel (no relocatable device
code), then linked into paper_2211_13295_gb300/libawe.so.  Rebuilds only what
changed.  Usage: python -m paper_2211_13295_gb300.build [--force]
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libawe.so")
SOURCES = ["awe_api.cu", "awe_bc.cu", "awe_recon.cu", "awe_predict.cu", "awe_flux.cu",
           "awe_gate.cu", "awe_tables.cu", "awe_peaks.cu", "awe_noalloc.cu", "awe_rk.cu"]
HEADERS = ["awe_internal.cuh", "fp_bits.cuh", "awe_flux.cuh", "awe_rk.h", "awe_tables.h", "awe_gate.h", "predict_index.cuh", "stencils.inc"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without FMA contraction, so that host-side tables round the same
# way on x86-64 and AArch64
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-Xptxas", "-O3"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _hdr_mtime():
    inc = os.path.join(os.path.dirname(HERE), "include", "awe.h")
    return max(os.path.getmtime(p) for p in [os.path.join(CSRC, h) for h in HEADERS] + [inc])


def _compile(src, force, extra):
    obj = os.path.join(OBJ, src.replace(".cu", ".o"))
    s = os.path.join(CSRC, src)
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), _hdr_mtime()):
        return obj
    cmd = [_nvcc()] + ARCH + FLAGS + extra + ["-c", s, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, extra), SOURCES))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
