"""Build the CUDA library ``libcrp.so`` in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel; the binary64 propagate
kernels are compiled with ``-fmad=false`` so that every multiply and add is
rounded separately, in source order.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcrp.so")
ROOT = os.path.dirname(HERE)

UNITS = {
    "api.cu": [],
    "field.cu": [],
    "tables.cu": [],
    "propagate_fp64.cu": ["-fmad=false"],
    "propagate_mixed.cu": [],
    "propagate_gmf.cu": [],
    "propagate_fixed.cu": [],
    "propagate_nuc_fp64.cu": ["-fmad=false"],
    "propagate_nuc_mixed.cu": [],
    "propagate_1d.cu": ["-fmad=false"],
    "hist_noalloc.cu": [],
    "lens.cu": [],
    "mlp.cu": [],
    "mlp_tc.cu": [],
    "peaks.cu": [],
}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "-Xcompiler", "-ffp-contract=off",
          "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcrp")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "crp.h"))
    cc = nvcc()
    jobs = []
    for unit, extra in UNITS.items():
        src = os.path.join(SRC, unit)
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        if force or _stale(obj, [src] + headers):
            cmd = [cc] + ARCH + COMMON + extra + ["-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose and r.stderr:
                print(r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    objs = [os.path.join(OUT, u.replace(".cu", ".o")) for u in UNITS]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcufft", "-Xlinker",
                                                             f"-rpath={cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
