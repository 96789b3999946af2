"""Builds the CUDA library libddot.so in-tree for sm_103a with nvcc.

The translation units are compiled in parallel and linked into
paper_2001_10986_gb300/_build/libddot.so (static CUDA runtime).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libddot.so")
SOURCES = ["dd_kernels.cu", "dd_api.cu", "dd_noalloc.cu", "dd_mlp.cu", "dd_glue.cu", "dd_gluing.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "dd.h"), __file__]
    return os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)


def build(verbose: bool = False, extra_flags=(), force: bool = False) -> str:
    """Compile libddot.so unless it is newer than every source (or force)."""
    if not force and not extra_flags and _up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    tmp = LIB + ".tmp"
    logs.append(_run([nvcc, *ARCH, "-shared", "-o", tmp, *objs]))
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force=True))
