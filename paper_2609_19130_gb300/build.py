"""Build libibf.so (sm_103a) in-tree with nvcc: the translation units compiled in parallel.

Beside it, libibf_probe.so: the fp64-pipe throughput probe that bench.py uses as the
denominator of the fp64 path's roofline (not part of the projection library)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libibf.so")
PROBE_LIB = os.path.join(OUT_DIR, "libibf_probe.so")
PROBE_SOURCE = "ibf_probe.cu"
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
SOURCES = ["ibf_kernels.cu", "ibf_yz.cu", "ibf_viscous.cu", "ibf_capi.cpp", "ibf_noalloc.cu"]
HEADERS = ["ibf_device.cuh", "ibf_common.cuh", "ibf_internal.h", "ibf_viscous.h", "tw96.inc"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return True
    if os.path.getmtime(PROBE_LIB) < os.path.getmtime(os.path.join(CSRC, PROBE_SOURCE)):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "ibf.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tw = os.path.join(CSRC, "tw96.inc")
    if not os.path.exists(tw):
        subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_twiddles.py")])

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu"] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PROBE_SOURCE]))
    for lib, o in ((LIB, objs[:-1]), (PROBE_LIB, objs[-1:])):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + o + ["-lcudart"])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
