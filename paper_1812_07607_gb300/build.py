"""Build the C-ABI library libdlsimjoin.so from csrc/ for sm_103a (in-tree).

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library next to this file (git-ignored). The CUDA runtime is linked
statically so the library loads without a CUDA library path; the driver API
entry points (tensor-map encoding) are fetched at run time.

    python -m paper_1812_07607_gb300.build [--ptxas-v] [--checked]
        --ptxas-v: print registers and spills
        --checked: the bounds-checked build (-DDL_CHECKED), libdlsimjoin_checked.so beside the
                   normal library: computed shared/global indices of the hot kernels are checked,
                   a failed check skips the access and is recorded (dl_debug_check_word)
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdlsimjoin.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libdlsimjoin_checked.so")

SOURCES = ["store.cu", "api.cu", "join_tc.cu", "join_simt.cu", "recheck.cu", "topk.cu", "noalloc.cu", "batch.cu", "server.cu", "tune.cu", "hist.cu", "cc.cu", "prune.cu", "hist_topk.cu"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, extra, bdir: str = BUILD) -> tuple[str, str]:
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(srcs, lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "dl.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile and link the library if any source is newer than it. Returns its path.

    checked=True builds the bounds-checked variant (-DDL_CHECKED) into its own library."""
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    extra = list(extra) + (["-DDL_CHECKED"] if checked else [])
    if not force and (checked or not extra) and not _stale(SOURCES, lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra), bdir), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []
    print(build(force=True, verbose=True, extra=extra, checked="--checked" in sys.argv))
