"""Builds libtsm.so in-tree for sm_103a (GB300).

Steps: run the code generator into ``_build/gen``; compile every
``csrc/*.cu`` and generated ``.cu`` with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) in parallel, skipping objects
newer than their sources and headers; link the shared library with the
shared CUDA runtime (the same libcudart PyTorch loads).

Usage:  python -m paper_1905_03136_gb300.build [--force] [-j N]
"""

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj")
LIB = os.path.join(PKG, "libtsm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(obj, src, deps_mtime):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < deps_mtime


def _compile(src, obj, extra):
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-6000:]))
    os.replace(obj + ".tmp", obj)
    return src, r.stderr


def build(force=False, jobs=None, verbose=False, ptxas_verbose=False):
    from . import codegen
    os.makedirs(OBJ, exist_ok=True)
    gen_files = codegen.generate(GEN)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu"))) + sorted(gen_files)
    hdr = _headers()
    deps_mtime = max([os.path.getmtime(h) for h in hdr] + [0])
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    todo = []
    objs = []
    for src in sources:
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or ptxas_verbose or _stale(obj, src, deps_mtime):
            todo.append((src, obj))
    jobs = jobs or max(1, min(len(todo) or 1, os.cpu_count() or 4))
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(jobs) as ex:
            futs = [ex.submit(_compile, s, o, extra) for s, o in todo]
            for f in cf.as_completed(futs):
                src, err = f.result()
                logs[src] = err
                if verbose:
                    print("compiled", os.path.relpath(src, ROOT), flush=True)
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-lcuda"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-4000:]))
        os.replace(tmp, LIB)
    return LIB, logs


def main():
    ap = argparse.ArgumentParser(description="build libtsm.so for sm_103a")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=None)
    ap.add_argument("--ptxas-verbose", action="store_true", help="print -Xptxas -v register/spill report")
    args = ap.parse_args()
    lib, logs = build(args.force, args.j, verbose=True, ptxas_verbose=args.ptxas_verbose)
    if args.ptxas_verbose:
        for src, err in sorted(logs.items()):
            print("==", os.path.relpath(src, ROOT))
            print(err)
    print(lib)


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    main()
