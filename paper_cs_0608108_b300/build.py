"""Build the CUDA library (libsi.so) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled to an object of its own (in
parallel, into _build/ at the repository root), then the objects are linked
into libsi.so.  An object is rebuilt when its source, or any header of csrc/
or include/, is newer than it.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build")
SO = os.path.join(PKG, "libsi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-Xcompiler", "-fPIC", "-std=c++17", "-O3", "-lineinfo", *ARCH]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _obj(src: str) -> str:
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def _newer(path: str, deps) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(p) > t for p in deps)


def _stale() -> bool:
    return _newer(SO, sources() + _headers())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    """Compile every .cu under csrc/ and link libsi.so (skipped when up to date)."""
    if not force and not _stale():
        return SO
    os.makedirs(OBJ, exist_ok=True)
    hdr = _headers()
    todo = [s for s in sources() if force or _newer(_obj(s), [s] + hdr)]

    def compile_one(src):
        cmd = [nvcc(), "-c", *FLAGS, f"-I{INCLUDE}", f"-I{CSRC}", "-o", _obj(src) + ".tmp", src]
        if ptxas_v:
            cmd[1:1] = ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}{r.stderr}")
        if (verbose or ptxas_v) and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        os.replace(_obj(src) + ".tmp", _obj(src))

    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 4))) as ex:
        list(ex.map(compile_one, todo))
    link = [nvcc(), "-shared", *ARCH, "-o", SO + ".tmp", *[_obj(s) for s in sources()], "-lcudart"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.check_call(link)
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv)
    print(SO)
