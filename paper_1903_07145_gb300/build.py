"""Build libipt.so in-tree for sm_103a (GB300).

Each translation unit compiles in parallel; the host scene builder goes
through g++ without floating-point contraction, the kernels through nvcc with
``-gencode arch=compute_103a,code=sm_103a``.  Objects land in ``_build/``
next to this file; the library is ``libipt.so`` in the package directory.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libipt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stderr


def _newest_input():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = sources()
    nv = nvcc()
    cmds = []
    objs = []
    for f in cu:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        cmd = [nv, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-o", o, os.path.join(CSRC, f)]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        cmds.append(cmd)
    for f in cpp:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        cmds.append(["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off",
                     "-I", INCLUDE, "-I", "/usr/local/cuda/include", "-o", o,
                     os.path.join(CSRC, f)])
    with cf.ThreadPoolExecutor(max_workers=max(2, len(cmds))) as ex:
        logs = list(ex.map(_compile, cmds))
    if verbose or ptxas_info:
        for l in logs:
            if l:
                print(l, file=sys.stderr)
    tmp = LIB + ".tmp"
    _compile([nv, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=True, ptxas_info=a.ptxas_info))
