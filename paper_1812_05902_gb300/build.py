"""Build libpivbos.so (the CUDA library behind include/pivbos.h) and
libpivbos_testing.so (include/pivbos_testing.h: checking and measurement
hooks that link the product library) in-tree.

Each translation unit is compiled for sm_103a only, in parallel, then linked
into ``paper_1812_05902_gb300/libpivbos.so``; ``testing.cu`` is linked on its
own against it.
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
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpivbos.so")
TESTING_LIB = os.path.join(HERE, "libpivbos_testing.so")
TESTING_SOURCES = ["testing.cu"]
SOURCES = ["api.cu", "medium.cu", "sort.cu", "render.cu", "render_batch.cu", "render_list.cu", "noalloc.cu", "batch.cu", "mlp.cu", "surrogate.cu", "bos.cu", "mie.cu", "pairs.cu", "selftest.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(ROOT, "include", h) for h in ("pivbos.h", "pivbos_testing.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    if (not force and os.path.exists(LIB) and os.path.exists(TESTING_LIB)
            and min(os.path.getmtime(LIB), os.path.getmtime(TESTING_LIB)) >= _deps()):
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    # measurement builds only (e.g. -DPIVBOS_DEPOSIT_AGG=0 for the unaggregated deposit)
    extra += os.environ.get("PIVBOS_NVCC_EXTRA", "").split()

    def compile_one(src):
        obj = os.path.join(OBJ, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + len(TESTING_SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES + TESTING_SOURCES))
    testing_objs = [o for o, _ in results[len(SOURCES):]]
    results = results[:len(SOURCES)]
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart", "-Xlinker", "-soname,libpivbos.so"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    tmp = TESTING_LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *testing_objs, "-L" + HERE, "-lpivbos", "-lcudart",
           "-Xlinker", "-rpath,$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("testing library link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, TESTING_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
