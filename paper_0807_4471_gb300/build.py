"""In-tree build of liblbgb.so (CUDA kernels + C ABI) for sm_103a.

The two translation units are compiled in parallel with nvcc and linked into
``paper_0807_4471_gb300/liblbgb.so``; objects go to ``paper_0807_4471_gb300/_build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbgb.so")
# (source, extra defines, object name); the step kernels are compiled once
# per storage precision so that the four compilations run in parallel.
UNITS = [("lb_kernels.cu", [f"-DLB_PREC={p}"], f"lb_kernels_p{p}.o") for p in range(4)] + [
    ("lb_dispatch.cu", [], "lb_dispatch.o"),
    ("lb_engine.cu", [], "lb_engine.o"),
    ("lb_api.cu", [], "lb_api.o"),
    ("lb_pool.cu", [], "lb_pool.o"),
    ("lb_noalloc.cu", [], "lb_noalloc.o"),
]
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["lb_internal.h", "lb_layout.cuh", "lb_engine.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbgb.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "lb.h"),
                                                                 os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblbgb.so if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src, defs, oname in UNITS:
        obj = os.path.join(BUILD, oname)
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, *defs, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            print(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
