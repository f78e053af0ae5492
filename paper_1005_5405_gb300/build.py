"""Build the sm_103a shared library libbz.so in-tree (nvcc, no cmake).

    python -m paper_1005_5405_gb300.build [--force] [--verbose]

The library lands in paper_1005_5405_gb300/_lib/libbz.so; build artefacts
are git-ignored.  The compile is one translation unit with one -gencode
(sm_103a), so it takes well under a minute.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libbz.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    srcs = [os.path.join(SRC, f) for f in sorted(os.listdir(SRC))]
    srcs.append(os.path.join(ROOT, "include", "bz.h"))
    return srcs


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    tmp = LIB + f".tmp{os.getpid()}"
    common = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              f"-I{os.path.join(ROOT, 'include')}", f"-I{SRC}"]
    if verbose:
        common.append("-Xptxas=-v")
    units = ["bz_api.cu", "bz_noalloc.cu", "bz_adjoint.cu"]
    objs = [os.path.join(OUT_DIR, u.replace(".cu", f".{os.getpid()}.o")) for u in units]
    # The translation units compile in parallel, then link into one library.
    procs = [subprocess.Popen(common + ["-c", "-o", o, os.path.join(SRC, u)],
                              stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for u, o in zip(units, objs)]
    outs = [p.communicate()[0] for p in procs]
    if any(p.returncode != 0 for p in procs):
        raise RuntimeError("nvcc failed:\n" + "\n".join(outs))
    if verbose:
        print("\n".join(outs))
    link = [nvcc, ARCH, "-shared", "-cudart", "shared",
            "-Xlinker", f"-rpath={os.path.join(cuda_home, 'lib64')}", "-o", tmp] + objs
    r = subprocess.run(link, capture_output=True, text=True)
    for o in objs:
        if os.path.exists(o):
            os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose))
