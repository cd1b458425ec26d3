"""Compile libh2bem.so in-tree for sm_103a (nvcc, one translation unit per
source file, compiled in parallel).  Host code is compiled without FMA
contraction so that the cluster tree's floating-point decisions follow the
written specification exactly on every host architecture."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libh2bem.so")
PEAKS = os.path.join(OUT_DIR, "peaks")  # arithmetic-peak microbenchmark (csrc/peaks.cu)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cpp", "gca.cpp", "hca.cpp", "k_gca.cu", "k_misc.cu", "k_nearsym.cu", "k_near_df.cu", "k_sing.cu", "k_sing_df.cu", "k_far.cu", "k_coupling.cu", "k_coupling_df.cu", "k_coupling_tc.cu", "k_cg.cu", "k_grad.cu", "k_grad_dlp.cu", "k_nearstore.cu", "k_hyper.cu", "k_p1.cu", "noalloc.cu"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _flags(src: str):
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        return ARCH + ["-lineinfo", "--expt-relaxed-constexpr", "-Xptxas", "-O3"] + common
    if src in ("gca.cpp", "hca.cpp"):  # the host constructions of the GCA / HCA bases run on OpenMP threads
        return common + ["-Xcompiler", "-fopenmp"]
    return common


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, "internal.h"), os.path.join(ROOT, "include", "h2bem.h")]
    headers += sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh"))
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc, *_flags(s), "-c", src, "-o", obj])
    psrc = os.path.join(CSRC, "peaks.cu")
    if force or _stale(PEAKS, [psrc]):
        jobs.append([nvcc, "-O3", *ARCH, psrc, "-o", PEAKS])
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    if any(j[-1] != PEAKS for j in jobs) or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "--cudart", "shared", "-o", tmp, *objs, "-lgomp"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
