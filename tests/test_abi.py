"""The C-ABI library builds, loads and exports every entry point of include/nys.h;
host-side argument validation rejects bad instances before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2510_04094_gb300 import build
    build.build()
    from paper_2510_04094_gb300 import _abi
    _abi.lib()
    return _abi


def _declared():
    src = open(os.path.join(ROOT, "include", "nys.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nys_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("nys_setup", "nys_assemble", "nys_solve", "nys_newton", "nys_grad", "nys_eval",
              "nys_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(abi):
    lib = abi.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(abi.EXPORTS) | {"nys_status_str", "nys_last_error"}


def test_struct_layout_matches_header(abi):
    assert C.sizeof(abi.nys_instance) == 16 + 8 * 4 + 32 + 64 + 16 + 8
    assert C.sizeof(abi.nys_options) == 24
    assert abi.nys_instance.t0.offset == 16 and abi.nys_instance.c.offset == 80
    assert abi.nys_instance.landmarks.offset == 144
    assert abi.nys_instance.bc.offset == 160 and abi.nys_instance.reserved.offset == 164


def _one(**kw):
    import nys_inputs as ni
    q = ni.cfg1()
    q.update(kw)
    return q


@pytest.mark.parametrize("bad", [dict(p=3), dict(n=2), dict(m=1), dict(m=230, n=300),
                                 dict(sigma=0.0), dict(gamma=-1.0), dict(t1=-1.0),
                                 dict(landmarks=[0, 5, 5] + list(range(6, 23))),
                                 dict(bc="bvp", p=1, a=[1.0], v=[0.0])])
def test_invalid_instances_are_rejected_on_the_host(abi, bad):
    from paper_2510_04094_gb300.api import pack_instances
    arr, keep = pack_instances([_one(**bad)])
    opt = abi.nys_options()
    ctx = C.c_void_p()
    code = abi.lib().nys_setup(C.byref(ctx), arr, 1, C.byref(opt), None)
    assert code == abi.NYS_EINVAL
    assert abi.lib().nys_last_error().decode().startswith("instance 0")
    assert not ctx.value


@pytest.mark.parametrize("kw,precision", [(dict(m=150), "mixed"),
                                          (dict(m=150, kind="nl", P=[0.0, -1.0, 0.0, 0.0]), "fp64")])
def test_large_landmark_counts_need_fp64_linear(abi, kw, precision):
    """Above NYS_M_MAX_MIXED landmarks only FP64 solves of the linear kinds run."""
    from paper_2510_04094_gb300.api import pack_instances
    arr, keep = pack_instances([_one(**kw)])
    opt = abi.nys_options()
    opt.precision = abi.NYS_MIXED if precision == "mixed" else abi.NYS_FP64
    ctx = C.c_void_p()
    assert abi.lib().nys_setup(C.byref(ctx), arr, 1, C.byref(opt), None) == abi.NYS_EINVAL
    assert "m > 112" in abi.lib().nys_last_error().decode()
    assert not ctx.value


@pytest.mark.parametrize("field,value", [("bc", 2), ("bc", -1), ("reserved", 1)])
def test_invalid_condition_fields_are_rejected_on_the_host(abi, field, value):
    from paper_2510_04094_gb300.api import pack_instances
    arr, keep = pack_instances([_one()])
    setattr(arr[0], field, value)
    opt = abi.nys_options()
    ctx = C.c_void_p()
    assert abi.lib().nys_setup(C.byref(ctx), arr, 1, C.byref(opt), None) == abi.NYS_EINVAL
    assert abi.lib().nys_last_error().decode().startswith("instance 0")
    assert not ctx.value


def test_status_strings(abi):
    for code in range(0, -10, -1):
        assert abi.lib().nys_status_str(code)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "nys.h"

int main(void) {
  /* every declaration of the header is visible to a plain C99 translation unit */
  int32_t (*fs)(nys_ctx**, const nys_instance*, int32_t, const nys_options*, void*) = nys_setup;
  int32_t (*fr)(nys_ctx*, void*, double*, int32_t*) = nys_run;
  if (!fs || !fr) return 3;
  nys_instance q;
  memset(&q, 0, sizeof q);
  q.p = 9;                       /* invalid order: rejected on the host, no device touched */
  nys_options opt;
  memset(&opt, 0, sizeof opt);
  nys_ctx* ctx = NULL;
  const int32_t r = nys_setup(&ctx, &q, 1, &opt, NULL);
  if (r != NYS_EINVAL || ctx != NULL) return 1;
  printf("%s|%s|%d|%d\n", nys_status_str(NYS_ENOTSPD), nys_last_error(), NYS_M_MAX,
         NYS_M_MAX_MIXED);
  return 0;
}
"""


def test_header_is_plain_c_and_links(abi, tmp_path):
    """include/nys.h compiles as C99 with warnings as errors, a C program links
    against libnys.so and gets host-side validation from it without a GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_nys.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_nys"
    libdir = os.path.dirname(abi._build.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lnys", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    status, err, mmax, mmix = out.stdout.strip().split("|")
    assert err.startswith("instance 0") and "p must be" in err
    assert int(mmax) == abi.NYS_M_MAX and int(mmix) == abi.NYS_M_MAX_MIXED
    assert status


def test_readme_c_example_compiles_and_links(abi, tmp_path):
    """The C usage example in README.md compiles (C99, -Werror) and links against
    libnys.so and the CUDA runtime (it needs a GPU to run)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if gcc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    readme = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", readme, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    libdir = os.path.dirname(abi._build.LIB_PATH)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.isdir(d)), None)
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), str(src), "-o", str(tmp_path / "example"),
           "-L", libdir, "-lnys", "-L", cudalib, "-lcudart", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_peak_probe_library_exports_its_header(abi, tmp_path):
    """include/nys_peak.h (the arithmetic-peak probes of the benchmark's roofline)
    compiles as C99 and libnys_peak.so exports what it declares; bad arguments are
    refused on the host."""
    import shutil
    import subprocess
    src = open(os.path.join(ROOT, "include", "nys_peak.h")).read()
    names = sorted(set(re.findall(r"\b(nys_[a-z_0-9]+)\s*\(", re.sub(r"/\*.*?\*/", "", src, flags=re.S))))
    assert names == ["nys_peak_launch"]
    lib = C.CDLL(abi._build.PEAK_LIB_PATH)
    for n in names:
        assert hasattr(lib, n)
    lib.nys_peak_launch.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    fl = C.c_double(-1.0)
    assert lib.nys_peak_launch(7, 10, None, None, C.byref(fl)) == -1
    assert lib.nys_peak_launch(0, 0, None, None, C.byref(fl)) == -1
    assert fl.value == -1.0
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    c = tmp_path / "peak.c"
    c.write_text('#include "nys_peak.h"\n'
                 'int main(void) {\n'
                 '  int32_t (*f)(int32_t, int32_t, void*, int32_t*, double*) = nys_peak_launch;\n'
                 '  return f ? 0 : 1;\n}\n')
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                    str(c), "-o", str(tmp_path / "peak.o")], check=True, capture_output=True)


def test_debug_build_links_and_exports_the_same_entry_points():
    """build(debug=True) (NYS_DEBUG_CHECKS) compiles every translation unit and
    links a library with the release library's entry points."""
    from paper_2510_04094_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libnys_debug.so") and os.path.exists(path)
    lib = C.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    status = open(os.path.join(ROOT, "include", "nys.h")).read()
    assert re.search(r"NYS_EBOUNDS\s*=\s*-10", status)
