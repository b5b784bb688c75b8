"""Build the CUDA library ``librtc.so`` in-tree with nvcc for sm_103a.

Usage: ``python -m paper_1903_01852_gb300.build [--force] [--ptxas-verbose]``.
Translation units are compiled in parallel; the library links the CUDA
runtime statically, so it needs only the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librtc.so")
SOURCES = ["rtc_kernels.cu", "rtc_runtime.cu", "rtc_server.cu", "rtc_noalloc.cu", "rtc_master.cu"]
HEADERS = [os.path.join(CSRC, "rtc_internal.h"), os.path.join(ROOT, "include", "rtc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librtc.so")


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True, defines=(), out=None) -> str:
    """Compile and link the library; ``defines`` adds -D tuning macros and ``out``
    names another output path (objects then go next to it)."""
    obj_dir = OBJ if out is None else os.path.join(os.path.dirname(os.path.abspath(out)), "_build")
    lib = LIB if out is None else os.path.abspath(out)
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include")]
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]
    common += [f"-D{d}" for d in defines]
    procs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or ptxas_verbose or defines or _stale(o, [s, *HEADERS]):
            cmd = [cc, *common, "-c", s, "-o", o]
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + text)
        if text.strip() and (ptxas_verbose or not quiet):
            sys.stdout.write(text)
    if force or procs or _stale(lib, objs):
        tmp = lib + ".tmp"
        cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, ptxas_verbose="--ptxas-verbose" in sys.argv, quiet=False))
