"""Build libfracsolve.so (sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel into an object
file under _build/, then linked into lib/libfracsolve.so.  Rebuilds only
when a source or header is newer than the library.

A second library, lib/libfracsolve_testhooks.so, links the same objects
except the block SpGEMM and sliced-ELL conversions and the AMG, which are
compiled once more with FS_TEST_HOOKS: in that build environment variables
can force the SpGEMM's long-row and chunked paths, jagged slices and the
fused prolongation on small problems, so that GPU tests cover them.  Only that
test loads it; the product library reads no environment variable.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libfracsolve.so")
LIB_HOOKS = os.path.join(LIBDIR, "libfracsolve_testhooks.so")
HOOKED = ("sparse.cu", "amg.cu")   # the translation units with test hooks
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_HOOKS)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_HOOKS))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    extra = extra or []

    def one(job):
        src, hooks = job
        base = os.path.basename(src).replace(".cu", "_hooks.o" if hooks else ".o")
        obj = os.path.join(BUILD, base)
        cmd = [cc, *ARCH, *FLAGS, *extra, *(["-DFS_TEST_HOOKS"] if hooks else []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    srcs = _sources()
    jobs = [(s, False) for s in srcs] + [(s, True) for s in srcs if os.path.basename(s) in HOOKED]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(one, jobs))
    plain = objs[:len(srcs)]
    hooked = [o for o, (s, _) in zip(plain, jobs) if os.path.basename(s) not in HOOKED] + objs[len(srcs):]
    for out, parts in ((LIB, plain), (LIB_HOOKS, hooked)):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *parts, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
