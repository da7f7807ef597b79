"""In-tree build of the bamg CUDA library (libbamg.so) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library under ``paper_2103_07537_gb300/_build/``.  Rebuilds only what
is older than its sources.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libbamg.so")
SOURCES = ["k_solve.cu", "k_sweep.cu", "k_ilu.cu", "k_schwarz.cu", "k_staged.cu", "k_setup.cu", "k_krylov.cu", "k_batched.cu", "k_transfer.cu", "k_learned.cu", "k_fields.cu", "k_dense_tc.cu", "k_pad.cu",
           "capi.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the bamg CUDA library cannot be built")
    return cand


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    return hs


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    hdr_time = max(os.path.getmtime(h) for h in _headers())
    procs = []
    objs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        fresh = (os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(sp)
                 and os.path.getmtime(obj) >= hdr_time)
        if force or not fresh:
            cmd = [nvcc()] + ARCH + NVCC_FLAGS + ["-c", sp, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), obj, cmd))
    failed = []
    for p, obj, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        else:
            os.replace(obj + ".tmp", obj)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    newest_obj = max(os.path.getmtime(o) for o in objs)
    if force or procs or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest_obj:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
