"""Builds libbpx.so in-tree with nvcc for sm_103a (GB300).

Usage: ``python -m paper_1904_11563_gb300.build`` or ``build()`` from Python.
Each translation unit compiles in its own nvcc process (in parallel); the
objects go to ``_build/`` beside this file and the shared library next to the
package's Python files.  A unit is recompiled unless its object carries the
SHA-256 of everything that went into it: the unit's text, every header's
text, the compiler flags, the nvcc release and the host machine type (so an
object built on another machine or from other sources is never linked).  The
library is relinked unless it carries the hash of its objects' hashes.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbpx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA 13 toolkit required)")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                   "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _compile(src, obj, verbose, extra):
    cmd = [_nvcc(), *(_flags()), *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def _nvcc_version() -> str:
    r = subprocess.run([_nvcc(), "--version"], capture_output=True, text=True)
    return r.stdout.strip().splitlines()[-1] if r.stdout.strip() else "unknown"


def _read_hash(path):
    try:
        with open(path) as f:
            return f.read().strip()
    except OSError:
        return None


def _write_hash(path, h):
    with open(path, "w") as f:
        f.write(h + "\n")


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> str:
    """Compiles every CUDA/C++ source of the package into libbpx.so; returns
    its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    common = hashlib.sha256()
    for part in (*_flags(), *extra_flags, _nvcc_version(), platform.machine(), sys.platform):
        common.update(part.encode() + b"\0")
    for hdr in sorted(_headers()):
        with open(hdr, "rb") as f:
            common.update(os.path.basename(hdr).encode() + b"\0" + f.read() + b"\0")
    jobs, objs, hashes = [], [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        h = common.copy()
        with open(s, "rb") as f:
            h.update(f.read())
        digest = h.hexdigest()
        objs.append(o)
        hashes.append(digest)
        if force or not os.path.exists(o) or _read_hash(o + ".sha256") != digest:
            jobs.append((s, o, digest))
    logs = []
    if jobs:
        for _s, o, _d in jobs:  # a failed compile leaves no object that looks current
            if os.path.exists(o + ".sha256"):
                os.remove(o + ".sha256")
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(_compile, s, o, verbose, list(extra_flags)) for s, o, _d in jobs]
            for f in futs:
                logs.append(f.result())
        for _s, o, d in jobs:
            _write_hash(o + ".sha256", d)
    lib_digest = hashlib.sha256("".join(hashes).encode()).hexdigest()
    if jobs or not os.path.exists(LIB) or _read_hash(LIB + ".sha256") != lib_digest:
        if os.path.exists(LIB + ".sha256"):
            os.remove(LIB + ".sha256")
        cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        _write_hash(LIB + ".sha256", lib_digest)
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
