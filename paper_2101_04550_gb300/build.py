"""Build the elbm CUDA library in-tree: ``_build/libelbm.so`` for sm_103a.

One nvcc process per translation unit (run in parallel), then a shared-library
link.  Rebuilds only when a source or header is newer than the library, and
then recompiles only the translation units whose own dependencies (the .d
files nvcc writes next to each object) changed.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libelbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# nvcc runs from this directory with relative paths, so that the dependency
# files it writes stay valid when the tree is copied elsewhere
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join("..", "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the elbm CUDA library cannot be built")
    return path


def _inputs():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "elbm.h"), __file__])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _deps(dep_file: str):
    """Files listed in an nvcc dependency file (make syntax), or None."""
    try:
        with open(dep_file) as fh:
            text = fh.read().replace("\\\n", " ")
    except OSError:
        return None
    _, _, rhs = text.partition(":")
    return [t for t in rhs.split() if t]


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = _deps(obj[:-2] + ".d")
    if deps is None:
        return True
    t = os.path.getmtime(obj)
    paths = [d if os.path.isabs(d) else os.path.join(HERE, d) for d in deps] + [src, __file__]
    return any(not os.path.exists(d) or os.path.getmtime(d) > t for d in paths)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    procs = []
    objs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if not force and not extra_flags and not _stale(src, obj):
            continue
        rel_src, rel_obj = os.path.relpath(src, HERE), os.path.relpath(obj, HERE)
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-MD", "-MF", rel_obj[:-2] + ".d", "-c", rel_src, "-o", rel_obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, cwd=HERE)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"{src}:\n{text}")
        elif verbose and text.strip():
            print(text, file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
