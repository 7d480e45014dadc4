"""Build libnb.so (the CUDA library behind include/nb.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library under paper_1812_00367_gb300/_build/.  The CUDA runtime is
linked statically so the library has no load-time dependency beyond the
driver.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnb.so")
SOURCES = ["nb_api.cu", "nb_kernels.cu", "nb_eval_fp64.cu", "nb_eval_ex.cu", "nb_eval_fp32.cu",
           "nb_eval_fp32x.cu", "nb_probe.cu", "nb_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnb")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "nb.h"))
    files.append(os.path.join(ROOT, "include", "nb_probe.h"))
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          out_dir: str | None = None, defines: dict | None = None) -> str:
    """Compile libnb.so.  out_dir / defines build a variant elsewhere (e.g. a
    debug or tuning build: defines={"NB_EVAL_MIN_BLOCKS": 5})."""
    out = out_dir or OUT
    lib = os.path.join(out, "libnb.so")
    os.makedirs(out, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    extra += [f"-D{k}={v}" for k, v in (defines or {}).items()]

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
