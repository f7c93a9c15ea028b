"""Build the sm_103a shared library librk.so in-tree with nvcc.

Usage: python -m paper_2412_16638_b300.build  (or build() from Python).
Each .cu file is compiled to an object in _build/ (in parallel), then linked
into paper_2412_16638_b300/librk.so with the CUDA runtime linked statically,
so the library loads on machines without a GPU.  Objects are rebuilt when
the source or any header in csrc/ or include/ is newer.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "librk.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _newest_header():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _deps_newer(obj):
    """True when a header recorded in obj's dependency file is newer than obj."""
    dep = obj[:-2] + ".d"
    if not os.path.exists(dep):
        return True
    t = os.path.getmtime(obj)
    text = open(dep).read().replace("\\\n", " ")
    for tok in text.split(":", 1)[-1].split():
        if tok.startswith("/usr/") or not os.path.exists(tok):
            continue
        if os.path.getmtime(tok) > t:
            return True
    return False


def _compile(src, obj, verbose):
    cmd = [NVCC] + ARCH + FLAGS + ["-MD", "-MF", obj[:-2] + ".d", "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return r.stderr


def build(verbose: bool = False, jobs: int = 8) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if verbose or not os.path.exists(o) or os.path.getmtime(o) < os.path.getmtime(s) or _deps_newer(o):
            todo.append((s, o))
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        for log in ex.map(lambda so: _compile(so[0], so[1], verbose), todo):
            if verbose and log:
                print(log, file=sys.stderr)
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
