"""Build libadg.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into one shared
library next to this file.  No cmake, no torch extension machinery: the
library is a plain C ABI (include/adg.h) over the CUDA runtime.
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
OUT = os.path.join(HERE, "libadg.so")
BUILD = os.path.join(HERE, "_build")
# The debug build (-DADG_DEBUG: bound checks in the kernels that record an
# error bit instead of accessing out of range), built on request only.
OUT_DEBUG = os.path.join(HERE, "libadg_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
SOURCES = ["adg_api.cu", "adg_kernels.cu", "adg_noalloc.cu", "adg_topo.cu", "adg_fd.cu", "adg_levels.cu", "adg_mesh.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "adg_internal.h"), os.path.join(CSRC, "adg_host.h"),
            os.path.join(ROOT, "include", "adg.h")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          debug: bool = False) -> str:
    bdir, lib_out = (BUILD_DEBUG, OUT_DEBUG) if debug else (BUILD, OUT)
    os.makedirs(bdir, exist_ok=True)
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, s.replace(".cu", ".o"))
        if force or _stale(obj, src):
            cmd = [nvcc(), *ARCH, *FLAGS, *(["-DADG_DEBUG"] if debug else []), "-c", src, "-o", obj]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out, file=sys.stderr)
    if jobs or not os.path.exists(lib_out) or force:
        tmp = lib_out + ".tmp%d" % os.getpid()
        cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcudart"]
        run(cmd)
        os.replace(tmp, lib_out)
    return lib_out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv,
                debug="--debug" in sys.argv))
