"""Build the CUDA library ``_lib/libocn.so`` in-tree for sm_103a (GB300).

Every translation unit is compiled in parallel with one ``-gencode`` and linked
against the shared CUDA runtime, so the process shares one runtime (and its
streams) with PyTorch.  Run ``python -m paper_2502_14148_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libocn.so")
SOURCES = ["capi.cu", "coeffs.cpp", "tendency_f64.cu", "tendency_f64_batch.cu"] + \
          [f"tendency_f32_r{r}{part}.cu" for r in (5, 3)
           for part in ("", "_smag", "_amd", "_batch", "_batch_smag", "_batch_amd")] + ["closure.cu",
           "poisson.cu", "reduce.cu", "noalloc.cu", "mlp.cu", "column.cu", "vertical.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libocn.so")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libocn.so; with checked=True the bounds-checked variant libocn_checked.so (every
    translation unit compiled with -DOCN_BOUNDS_CHECK=1, objects in _build_checked/)."""
    nvcc = _nvcc()
    obj_dir = OBJ + "_checked" if checked else OBJ
    lib_path = os.path.join(LIBDIR, "libocn_checked.so") if checked else LIB
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = [os.path.join(CSRC, "ocn_internal.cuh"), os.path.join(CSRC, "tendency_kernel.cuh"),
               os.path.join(CSRC, "column.cuh"), os.path.join(CSRC, "batch.cuh"),
               os.path.join(ROOT, "include", "ocn.h")]
    flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-I" + os.path.join(ROOT, "include")] + ARCH
    if verbose:
        flags += ["-Xptxas", "-v"]
    if checked:
        flags += ["-DOCN_BOUNDS_CHECK=1"]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
        if force or _newer(o, [s] + headers):
            jobs.append([nvcc] + flags + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for f, j in zip(futs, jobs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(j))
    objs = [os.path.join(obj_dir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    if force or jobs or _newer(lib_path, objs):
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = [nvcc, "-shared", "-cudart", "shared", "-o", tmp] + objs + ARCH + \
              ["-Xlinker", "-rpath=" + _cuda_lib_dir(nvcc)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
