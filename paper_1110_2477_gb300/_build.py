"""Build the CUDA library libob.so in-tree (sm_103a only).

The library is several translation units (the host side and small kernels in
ob_lib.cu, the induction kernels in their own units) compiled in parallel to
objects, then linked into one shared library.
"""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
UNITS = ["ob_lib.cu", "ob_batched16.cu", "ob_batched8.cu", "ob_batched_half.cu", "ob_tiers.cu", "ob_group.cu", "ob_greeks8.cu",
         "ob_greeks.cu", "ob_path.cu"]
SRC = [os.path.join(CSRC, u) for u in UNITS]
DEPS = SRC + [os.path.join(CSRC, f) for f in ("ob_kern.cuh", "ob_tc.cuh", "ob_team.cuh", "ob_adj.cuh", "ob_path.cuh")] + [
    os.path.join(ROOT, "include", "ob.h")]
LIB = os.path.join(HERE, "libob.so")
OBJ = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force=False, verbose=False):
    """Compile the library if it is missing or older than its sources."""
    if not force and os.path.exists(LIB):
        mt = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= mt for d in DEPS):
            return LIB
    os.makedirs(OBJ, exist_ok=True)
    tag = "%d" % os.getpid()
    objs = [os.path.join(OBJ, os.path.splitext(u)[0] + "." + tag + ".o") for u in UNITS]

    def compile_one(args):
        src, obj = args
        cmd = [nvcc()] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                 "-I" + os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        list(ex.map(compile_one, zip(SRC, objs)))
    tmp = LIB + ".tmp." + tag
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB
