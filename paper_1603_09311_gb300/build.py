"""Build libsdd.so in-tree with nvcc for sm_103a (GB300).

Six translation units compiled in parallel and linked into one shared
library with the static CUDA runtime:
  walk_f32.cu  single-precision walk  (-ftz=true -prec-div=false -prec-sqrt=false)
  walk_f64.cu  double-precision walk  (-fmad=false: no fused multiply-add)
  sdd_api.cu   C ABI, planning, reduction
  interp.cu    interpolation between Monte Carlo interface nodes (FP64)
  mt.cu        apparent resistivity and phase at measurement sites (FP64)
  rbffd.cu     RBF-FD sub-domain solve (FP64, -fmad=false)
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsdd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
UNITS = {
    "walk_f32": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "walk_f64": ["-fmad=false"],
    "sdd_api": [],
    "interp": [],
    "mt": [],
    "rbffd": ["-fmad=false"],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsdd")
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sdd.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not ptxas_info and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(BUILD, unit + ".o")
        cmd = [cc, *ARCH, *COMMON, *flags, "-c", os.path.join(CSRC, unit + ".cu"), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((unit, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs, failed = [], []
    for unit, obj, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if verbose or ptxas_info or p.returncode != 0:
            sys.stdout.write(text)
        if p.returncode != 0:
            failed.append(unit)
        objs.append(obj)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + ".tmp"
    subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True, ptxas_info="-v" in sys.argv)
