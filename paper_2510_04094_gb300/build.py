"""Build the C-ABI shared library libnys.so (sm_103a) in-tree.

Each CUDA translation unit is compiled by its own nvcc process (in parallel),
then linked with the shared CUDA runtime so that the library shares the
runtime instance of the host process (PyTorch's, when it is loaded first).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
INC_DIR = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libnys.so")
SOURCES = ["nys_setup.cu", "nys_assemble.cu", "nys_assemble_tc.cu", "nys_solve.cu", "nys_eval.cu",
           "nys_newton.cu",
           "nys_grad.cu", "nys_noalloc.cu", "nys_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC_DIR, "-I" + SRC_DIR]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile every .cu in csrc/ for sm_103a and link _lib/libnys.so. Returns the path."""
    nvcc = _nvcc()
    os.makedirs(OBJ_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    headers = [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR) if f.endswith(".cuh")]
    headers.append(os.path.join(INC_DIR, "nys.h"))
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(SRC_DIR, s))]
    jobs = []
    for s in srcs:
        src = os.path.join(SRC_DIR, s)
        obj = os.path.join(OBJ_DIR, s + ".o")
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc] + ARCH + FLAGS + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OBJ_DIR, s + ".o") for s in srcs]
    if force or jobs or not os.path.exists(LIB_PATH):
        cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
        tmp = LIB_PATH + ".tmp"
        run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
            + ["-Xlinker", "-rpath=" + cudalib])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
