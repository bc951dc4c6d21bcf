"""Build libigks.so in-tree for sm_103a with nvcc (one -gencode, translation units
compiled in parallel, then linked). Used by __graft_entry__.build() and on first import
of the binding when the library is missing or older than its sources."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libigks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
# per translation unit: the cell kernels round every product before adding (see igks_cell.cu)
PER_FILE = {"igks_cell.cu": ["-fmad=false"], "igks_noalloc.cu": ["-fmad=false"]}
_lock = threading.Lock()


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        objs, procs = [], []
        for src in sources():
            obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc(), *ARCH, *FLAGS, *PER_FILE.get(os.path.basename(src), []), *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
            objs.append(obj)
        failed = []
        for p, src in procs:
            out, _ = p.communicate()
            if verbose or p.returncode:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode:
                failed.append(src)
        if failed:
            raise RuntimeError(f"nvcc failed on {failed}")
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
