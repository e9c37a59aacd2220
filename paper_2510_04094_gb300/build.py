"""Build the C-ABI shared libraries (sm_103a) in-tree: libnys.so, the solver
(include/nys.h), and libnys_peak.so, the arithmetic-peak probes that the
benchmark divides by (include/nys_peak.h).

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
PEAK_LIB_PATH = os.path.join(LIB_DIR, "libnys_peak.so")
DEBUG_LIB_PATH = os.path.join(LIB_DIR, "libnys_debug.so")
SOURCES = ["nys_setup.cu", "nys_assemble.cu", "nys_assemble_tc.cu", "nys_assemble_band.cu",
           "nys_solve.cu", "nys_refine_band.cu", "nys_eval.cu", "nys_newton.cu", "nys_grad.cu",
           "nys_noalloc.cu", "nys_api.cu"]
PEAK_SOURCES = ["nys_peak.cu"]
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


def build(force=False, verbose=False, debug=False):
    """Compile the .cu sources for sm_103a and link _lib/libnys.so and
    _lib/libnys_peak.so.  Returns the solver library's path.

    debug=True builds _lib/libnys_debug.so instead (objects in _build_debug/):
    the same solver with NYS_DEBUG_CHECKS, whose kernels check their shared-
    and global-memory indices, skip a failing access and report NYS_EBOUNDS
    for the instance (see include/nys.h)."""
    nvcc = _nvcc()
    obj_dir = OBJ_DIR + ("_debug" if debug else "")
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    headers = [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR) if f.endswith(".cuh")]
    headers += [os.path.join(INC_DIR, f) for f in os.listdir(INC_DIR) if f.endswith(".h")]
    if debug:
        libs = [(DEBUG_LIB_PATH, SOURCES)]
        flags = FLAGS + ["-DNYS_DEBUG_CHECKS"]
    else:
        libs = [(LIB_PATH, SOURCES), (PEAK_LIB_PATH, PEAK_SOURCES)]
        flags = FLAGS
    jobs = []
    for _, sources in libs:
        for s in sources:
            src = os.path.join(SRC_DIR, s)
            obj = os.path.join(obj_dir, s + ".o")
            if force or _stale(obj, [src] + headers):
                jobs.append([nvcc] + ARCH + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            list(ex.map(run, jobs))
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    for path, sources in libs:
        objs = [os.path.join(obj_dir, s + ".o") for s in sources]
        if force or not os.path.exists(path) or any(os.path.getmtime(o) > os.path.getmtime(path)
                                                    for o in objs):
            tmp = path + ".tmp"
            run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
                + ["-Xlinker", "-rpath=" + cudalib])
            os.replace(tmp, path)
    return libs[0][0]


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
