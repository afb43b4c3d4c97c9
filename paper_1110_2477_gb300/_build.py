"""Build the CUDA library libob.so in-tree (sm_103a only)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "ob_lib.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("ob_tc.cuh", "ob_team.cuh", "ob_adj.cuh")] + [
    os.path.join(ROOT, "include", "ob.h")]
LIB = os.path.join(HERE, "libob.so")


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
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"), "-o", tmp] + SRC
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB
