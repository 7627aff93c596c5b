"""Builds libptycho.so in place (nvcc, sm_103a) from csrc/, and with
--checked the checked build libptycho_checked.so (PTYCHO_CHECKED=1: index
checks in the kernels, reported by ptycho_check as PTYCHO_ECHECK).

Usage: python -m paper_2505_14372_b300.build [-j JOBS] [--force] [--checked]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libptycho.so")
OBJ_CHECKED = os.path.join(HERE, "_build", "checked")
LIB_CHECKED = os.path.join(HERE, "libptycho_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++20", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", SRC, "-I", INC]


def sources():
    return sorted(f for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def headers_mtime():
    hs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INC, f) for f in os.listdir(INC)]
    return max(os.path.getmtime(h) for h in hs)


def compile_one(src, force, hmt, objdir=OBJ, defines=()):
    obj = os.path.join(objdir, src + ".o")
    path = os.path.join(SRC, src)
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), hmt):
        return obj, ""
    cmd = [NVCC, *ARCH, *COMMON, *defines, "-c", path, "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["-x", "cu"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(jobs: int = 8, force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    objdir, lib = (OBJ_CHECKED, LIB_CHECKED) if checked else (OBJ, LIB)
    defines = ["-DPTYCHO_CHECKED=1"] if checked else []
    os.makedirs(objdir, exist_ok=True)
    hmt = headers_mtime()
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: compile_one(s, force, hmt, objdir, defines), sources()))
    newest = max(os.path.getmtime(o) for o, _ in objs)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        cmd = [NVCC, *ARCH, "-shared", "-o", lib, *[o for o, _ in objs], "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        for o, log in objs:
            if log:
                print(log)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=8)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", action="store_true")
    ap.add_argument("--checked", action="store_true", help="build libptycho_checked.so")
    a = ap.parse_args()
    print(build(a.j, a.force, a.v, a.checked))
    sys.exit(0)
