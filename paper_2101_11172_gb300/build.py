"""Build the CUDA library in-tree: ``paper_2101_11172_gb300/_build/libws_gb300.so``.

sm_103a only (``-gencode arch=compute_103a,code=sm_103a``); host sources are
portable C++17 (no architecture-specific flags), so the same command builds on
x86-64 and on aarch64.  Translation units compile in parallel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libws_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["wstack.cu", "transforms.cu", "transforms_4096.cu", "transforms_2048.cu", "transforms_small.cu",
              "noalloc.cu", "fp64.cu"]
CXX_SOURCES = ["plan.cpp", "lmfit.cpp", "batch.cpp", "tune.cpp"]


def cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    out = [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh"))]
    out.append(os.path.join(ROOT, "include", "ws.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    inc = ["-I" + os.path.join(home, "include"), "-I" + os.path.join(ROOT, "include")]
    os.makedirs(BUILD, exist_ok=True)
    jobs, objs = [], []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", *inc,
               "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    procs = [(subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), c) for c, _ in jobs]
    failed = []
    for pr, c in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((c, out.decode(errors="replace")))
        elif verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("building libws_gb300 failed:\n" + msg)
    objs = [o for _, o in jobs]
    libdir = os.path.join(home, "lib64")
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs,
            "-Xlinker", "-rpath=" + libdir]
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
