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
