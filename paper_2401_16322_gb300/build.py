"""Build the in-tree CUDA library ``libewave.so`` for sm_103a.

Compiles the translation units under ``csrc/`` in parallel with nvcc (one ``-gencode``),
then links them into ``paper_2401_16322_gb300/libewave.so``.  No torch extension machinery:
the library exposes a plain C ABI (``include/ewave.h``) that the Python binding loads with
ctypes.  Usage: ``python -m paper_2401_16322_gb300.build [--verbose]``.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libewave.so")
BUILD_DIR = os.path.join(ROOT, "_build")
SOURCES = ["kernels_stencil.cu", "kernels_aux.cu", "kernels_tma.cu", "kernels_3d.cu",
           "kernels_tma3d.cu", "kernels_kadj.cu", "kernels_mgs.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libewave.so")


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return r


def build(verbose=False, ptxas_verbose=False):
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]
    objs = []
    jobs = []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        jobs.append([nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda c: _run(c, verbose or ptxas_verbose), jobs))
    if ptxas_verbose:
        for r in results:
            sys.stdout.write(r.stderr)
    tmp = OUT + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], verbose)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, ptxas_verbose="--ptxas" in sys.argv)
    print(OUT)
