"""Build the sm_103a shared library in-tree with nvcc (no cmake, no torch JIT).

Three translation units compile in parallel, then link into
``paper_1703_00185_gb300/libd2q37_gb300.so``.  Host code is compiled with
``-ffp-contract=off`` so the host-side initial-state recipe rounds the same
way on every machine.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libd2q37_gb300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
SOURCES = ["d2q37_kernels.cu", "d2q37_kernels_fp32.cu", "d2q37_api.cu", "d2q37_batch.cu", "d2q37_batch_static.cu", "d2q37_server.cu", "quadrature_dd.cu"]
HEADERS = ["d2q37_lattice.cuh", "d2q37_launch.h", "d2q37_handle.h", "dfloat.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the D2Q37 library")
    return path


def _flags(src):
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + os.path.join(HERE, "..", "include")]
    if not src.endswith(".cu"):
        return common + ["-x", "c++"]
    flags = common + ARCH + ["-lineinfo"] + os.environ.get("D2Q37_NVCC_FLAGS", "").split()
    if os.environ.get("D2Q37_PTXAS_V"):
        flags += ["-Xptxas", "-v"]
    return flags


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "d2q37.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile and link the library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(OBJ_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ_DIR, src + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
