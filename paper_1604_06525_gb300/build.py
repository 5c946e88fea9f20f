"""In-tree build of the CUDA solver library for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel and linked
into paper_1604_06525_gb300/_lib/libopt_gb300.so; nothing is installed.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
BUILDDIR = os.path.join(ROOT, "_build")
LIBNAME = "libopt_gb300.so"
SOURCES = ["api.cu", "batch.cu", "grid_kernels.cu", "graph_kernels.cu", "graph2d_kernels.cu", "materialize.cu",
           "noalloc.cu", "serve.cu", "fp64.cu",
           "embedded_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver library")
    return cand


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, defines=()) -> str:
    """Compile and link the library if a source changed; returns its path.
    defines: extra preprocessor definitions ("NAME=value"), for measuring
    compile-time variants of a kernel (pass force=True)."""
    out = lib_path()
    if not force and not _stale(out):
        return out
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILDDIR, exist_ok=True)
    nvcc = nvcc_path()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC]
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    common += [f"-D{d}" for d in defines]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILDDIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"--- {src} ---\n{log.decode(errors='replace')}")
        elif verbose or ptxas_info:
            sys.stderr.write(log.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = out + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
