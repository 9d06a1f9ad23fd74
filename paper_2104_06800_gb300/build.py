"""Build the CUDA library in-tree: every csrc/*.cu is compiled for sm_103a in
parallel and linked into libvoldor_em.so next to this file.

Usage: python -m paper_2104_06800_gb300.build [--force]
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvoldor_em.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build the library)")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest(extra):
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    h.update(" ".join(extra).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


CHECKED_LIB = os.path.join(HERE, "libvoldor_em_checked.so")


def build(force: bool = False, verbose: bool = False, extra_flags=(), lib_path: str | None = None,
          build_dir: str | None = None, checked: bool = False) -> str:
    """Compile (if sources changed) and return the path of the shared library.

    extra_flags: additional nvcc flags (for example -D options of the kernels);
    lib_path / build_dir: where to put the library and the objects;
    checked: the index-checking build (-DVD_CHECKED) as libvoldor_em_checked.so."""
    if checked:
        extra_flags = (*extra_flags, "-DVD_CHECKED")
        lib_path = lib_path or CHECKED_LIB
        build_dir = build_dir or os.path.join(HERE, "_build_checked")
    LIB = lib_path or globals()["LIB"]
    BUILD = build_dir or globals()["BUILD"]
    flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
             *ARCH, *extra_flags]
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest(flags)
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
