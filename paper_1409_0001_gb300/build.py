"""In-tree build of the CUDA library (libcgdiff.so) for GB300 (sm_103a).

Every translation unit under csrc/ is compiled in parallel with nvcc and linked into
one shared library next to this file.  No cmake, no torch extension machinery:
the library has a plain C ABI (include/cg.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(HERE, "libcgdiff.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max([os.path.getmtime(h) for h in hs] + [0.0])


def _compile(src: str, extra):
    """Compile one source unless its object is newer than it and every header;
    returns (object path, whether nvcc ran)."""
    obj = os.path.join(BUILD_DIR, os.path.basename(src)[:-3] + ".o")
    if (os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
            and os.path.getmtime(obj) >= _headers_mtime()):
        return obj, False
    cmd = [_nvcc()] + NVCC_FLAGS + ARCH + list(extra) + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
    if res.stderr.strip():
        sys.stderr.write(res.stderr)
    return obj, True


def build(force: bool = False, extra=(), verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libcgdiff.so; returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = sources()
    if force:
        for s in srcs:
            o = os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o")
            if os.path.exists(o):
                os.remove(o)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        done = list(ex.map(lambda s: _compile(s, extra), srcs))
    objs = [o for o, _ in done]
    compiled = [os.path.basename(s) for s, (_, ran) in zip(srcs, done) if ran]
    newest = max(os.path.getmtime(o) for o in objs)
    linked = force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest
    if linked:
        tmp = LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = [_nvcc(), "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
        os.replace(tmp, LIB_PATH)
    if verbose:
        print("built %s: compiled %s; reused %d object(s); %s" % (
            LIB_PATH, ", ".join(compiled) if compiled else "nothing",
            len(objs) - len(compiled), "linked" if linked else "library up to date"))
    return LIB_PATH


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
