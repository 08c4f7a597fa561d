"""Build librs_b300.so (all CUDA sources of csrc/) for sm_103a with nvcc.

The library is built in-tree, next to this file, so that it travels with the
repository.  A hash of the sources is written beside it; the Python binding
refuses to load a library whose sources have changed since it was built.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librs_b300.so")
HASH = LIB + ".srchash"
# the bounds-checked library (RS_CHECKED: the shoot kernels check every
# count-map and window index before writing), built beside the library from
# the same objects with rs_shoot.cu compiled a second time
LIB_CHECKED = os.path.join(HERE, "librs_b300_checked.so")
CHECKED_SRC = "rs_shoot.cu"
BUILD_DIR = os.path.join(ROOT, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE,
                     "-Xptxas", "-warn-spills"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  glob.glob(os.path.join(CSRC, "*.cpp")))


def source_hash() -> str:
    h = hashlib.sha256()
    files = sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                               glob.glob(os.path.join(CSRC, "*.h"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h"))) + [os.path.abspath(__file__)]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _code_only(text: str) -> str:
    """C/C++ source without its comments and blank-space differences."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Hash of the code (comments excluded) that defines the deflection
    kernel: its profile figures stay valid while this is unchanged."""
    h = hashlib.sha256()
    for f in (os.path.join(CSRC, "rs_shoot.cu"), os.path.join(CSRC, "rs_internal.cuh"),
              os.path.join(INCLUDE, "rs.h")):
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librs_b300.so")
    return cand


def _compile(src: str, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(BUILD_DIR, os.path.basename(src) + (".checked.o" if checked else ".o"))
    cmd = [nvcc(), *NVCC_FLAGS, *(["-DRS_CHECKED"] if checked else []), "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def _link(objs: list[str], lib: str) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source in csrc/ and link librs_b300.so and the
    bounds-checked librs_b300_checked.so (if stale)."""
    digest = source_hash()
    if not force and os.path.exists(LIB) and os.path.exists(LIB_CHECKED) and \
            os.path.exists(HASH):
        with open(HASH) as fh:
            if fh.read().strip() == digest:
                return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = sources()
    jobs = [(s, False) for s in srcs] + \
        [(s, True) for s in srcs if os.path.basename(s) == CHECKED_SRC]
    # the slowest compiles first
    jobs.sort(key=lambda j: os.path.basename(j[0]) != CHECKED_SRC)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    normal = [o for o, (_, c) in zip(objs, jobs) if not c]
    checked = [o for o, (s, c) in zip(objs, jobs)
               if c or os.path.basename(s) != CHECKED_SRC]
    _link(normal, LIB)
    _link(checked, LIB_CHECKED)
    with open(HASH, "w") as fh:
        fh.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
