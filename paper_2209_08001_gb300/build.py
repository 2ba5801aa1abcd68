"""In-tree build of libnks.so for sm_103a (nvcc, no cmake).

Each translation unit compiles in parallel; the shared library lands next to
this file, where the binding loads it.  ``python -m paper_2209_08001_gb300.build``
builds it by hand.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnks.so")
SOURCES = ["nks_stencil.cu", "nks_krylov.cu", "nks_ras.cu", "nks_api.cu", "nks_noalloc.cu", "nks_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "nks.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


# the sources each profiled kernel is compiled from (its own file, the headers it uses)
KERNEL_SOURCES = {
    "k_ras_apply_lane": ["nks_ras.cu", "nks_pattern.cuh", "nks_internal.cuh"],
    "k_ras_apply": ["nks_ras.cu", "nks_pattern.cuh", "nks_internal.cuh"],
    "k_jv32": ["nks_stencil.cu", "nks_model3.cuh", "nks_internal.cuh"],
}


def source_hash(kernel: str = None) -> str:
    """sha256 (16 hex digits) of the sources a kernel is compiled from (all of the
    library's when kernel is None or unknown), the C header and the build flags:
    identifies the kernel build a profile was taken of."""
    import hashlib
    h = hashlib.sha256()
    files = sorted(KERNEL_SOURCES.get(kernel) or os.listdir(CSRC))
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "include", "nks.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS[:3]).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s" % src)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("link of libnks.so failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv,
          extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ())
    print(LIB)
