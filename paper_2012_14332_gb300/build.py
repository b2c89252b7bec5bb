"""Compile the CUDA library ``libabc_gb300.so`` in-tree for sm_103a (nvcc only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libabc_gb300.so")
SOURCES = ["abc_kernels.cu", "abc_batch.cu", "abc_maf.cu", "abc_api.cu", "abc_plan.cu", "abc_smc.cu", "abc_pmc.cu"]
HEADERS = ["abc_kernels.h", "abc_model.cuh"]
PUBLIC_HEADER = os.path.join(os.path.dirname(HERE), "include", "abc_gb300.h")

# -fmad=false: no FMA contraction anywhere; the fast path asks for FMA
# explicitly (__fmaf_rn), the exact path must never get one.
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-shared"]


# The flow kernels are accurate to a tolerance (BF16 products), not bit for
# bit, and include no exact-mode model arithmetic: FMA contraction is allowed
# there.
FMAD_SOURCES = {"abc_maf.cu"}


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [PUBLIC_HEADER, __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Build the library if it is missing or older than its sources: every
    translation unit compiled in parallel, then one shared-library link."""
    if not force and not _stale():
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    procs = []
    for f in SOURCES:
        obj = os.path.join(objdir, f.replace(".cu", ".o"))
        flags = [x for x in NVCC_FLAGS if x != "-shared"]
        if f in FMAD_SOURCES:
            flags = ["-fmad=true" if x == "-fmad=false" else x for x in flags]
        cmd = [nvcc()] + flags + (["-Xptxas", "-v"] if verbose else []) + \
            ["-c", "-o", obj, os.path.join(CSRC, f)]
        procs.append((f, obj, subprocess.Popen(cmd, cwd=CSRC)))
    objs = []
    for f, obj, pr in procs:
        if pr.wait() != 0:
            raise RuntimeError("nvcc failed on %s" % f)
        objs.append(obj)
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
