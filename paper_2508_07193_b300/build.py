"""Build libflashmp.so in-tree with nvcc for sm_103a.

    python -m paper_2508_07193_b300.build [--force]

Objects go to ``paper_2508_07193_b300/_build``; the shared library lands next
to this file so that it ships with the source tree.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libflashmp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest(paths, flags):
    """SHA-256 of the files' contents and the compile flags."""
    h = hashlib.sha256(" ".join(flags).encode())
    for p in paths:
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _stale(target, digest):
    """The target is missing, or was built from other contents than those
    that give `digest` (recorded beside it): a shipped library newer than its
    sources is rebuilt all the same when they differ."""
    stamp = target + ".sha256"
    if not os.path.exists(target) or not os.path.exists(stamp):
        return True
    with open(stamp) as f:
        return f.read().strip() != digest


def _stamp(target, digest):
    with open(target + ".sha256", "w") as f:
        f.write(digest + "\n")


def build(force=False, verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    headers = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    headers.append(os.path.join(ROOT, "include", "flashmp.h"))
    jobs = []
    objs = []
    digests = {}
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        digests[obj] = _digest([src] + headers, ARCH + FLAGS + list(extra))
        if force or _stale(obj, digests[obj]):
            jobs.append(([nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj], obj))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    def compile_one(job):
        cmd, obj = job
        run(cmd)
        _stamp(obj, digests[obj])

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        list(ex.map(compile_one, jobs))
    lib_digest = hashlib.sha256("".join(digests[o] for o in objs).encode()).hexdigest()
    if force or jobs or _stale(LIB, lib_digest):
        # cuSOLVER: the set-up Cholesky of the compact-layout correction matrices
        run([nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcusolver"])
        _stamp(LIB, lib_digest)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    verbose = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=force, verbose=verbose or bool(extra), extra=extra))
