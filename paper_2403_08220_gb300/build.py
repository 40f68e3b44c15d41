"""Build the in-tree CUDA library `libdino.so` for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
`paper_2403_08220_gb300/_build/libdino.so` (static CUDA runtime).  Run as
`python -m paper_2403_08220_gb300.build` or call `build()`.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdino.so")
SOURCES = ["host.cpp", "k_reduced.cu", "k_woodbury.cu", "k_simt.cu", "k_tc.cu", "k_da.cu",
           "k_diag.cu", "k_eig.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(HERE, "..", "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdino")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "dino.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, extra_flags=None) -> str:
    """Compile every CUDA/C++ source and link libdino.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    flags = FLAGS + list(extra_flags or [])
    jobs = []
    for s in _sources():
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, s.rsplit(".", 1)[0] + ".o")
        lang = ["-x", "cu"] if s.endswith(".cpp") else []
        cmd = [nvcc] + ARCH + flags + lang + ["-c", src, "-o", obj]
        jobs.append((s, src, obj, cmd))

    def run(job):
        name, src, obj, cmd = job
        if not _stale(obj, src):
            return name, 0, ""
        p = subprocess.run(cmd, capture_output=True, text=True)
        return name, p.returncode, p.stdout + p.stderr

    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        results = list(ex.map(run, jobs))
    for name, rc, out in results:
        if verbose and out:
            print(f"[{name}]\n{out}", file=sys.stderr)
        if rc != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{out}")
    objs = [j[2] for j in jobs]
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
