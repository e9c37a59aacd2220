"""ctypes binding of include/nys.h: the same entry points under the same names.

Argument marshalling only -- every step of the solver runs in libnys.so.
Loading fails loudly when the library has not been built (there is no CPU
fallback).
"""
import ctypes as C
import os

from . import build as _build

NYS_OK, NYS_EINVAL, NYS_ENOMEM, NYS_ECUDA = 0, -1, -2, -3
NYS_ENOTSPD, NYS_ENOCONV, NYS_ENONFINITE, NYS_ETIMEOUT = -4, -5, -6, -7
NYS_EPRECISION, NYS_ESTATE = -8, -9
NYS_EBOUNDS = -10   # builds with NYS_DEBUG_CHECKS only
NYS_FP64, NYS_MIXED, NYS_MIXED_F64F = 0, 1, 2
NYS_ASM_AUTO, NYS_ASM_SIMT, NYS_ASM_TUNE, NYS_ASM_TC = 0, 1, 2, 3
NYS_COEF_TABLE, NYS_COEF_LIN, NYS_COEF_POLY_NL = 0, 1, 2
NYS_BC_IVP, NYS_BC_BVP = 0, 1
NYS_M_MAX = 224
NYS_M_MAX_MIXED = 112


class nys_instance(C.Structure):
    _fields_ = [("p", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("kind", C.c_int32),
                ("t0", C.c_double), ("t1", C.c_double), ("sigma", C.c_double),
                ("gamma", C.c_double), ("v", C.c_double * 4), ("c", C.c_double * 8),
                ("landmarks", C.POINTER(C.c_int32)), ("coef_table", C.POINTER(C.c_double)),
                ("bc", C.c_int32), ("reserved", C.c_int32)]


class nys_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("refine_steps", C.c_int32), ("eig_tau", C.c_double),
                ("scale_sqrt_m", C.c_int32), ("assembly", C.c_int32)]


class NysError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (lib().nys_status_str(code).decode(), code, msg))
        self.code = code


_LIB = None


def lib():
    """Load libnys.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError("libnys.so is not built (%s); run paper_2510_04094_gb300.build.build()"
                               % path)
        L = C.CDLL(path)
        vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
        L.nys_setup.argtypes = [C.POINTER(vp), C.POINTER(nys_instance), i32, C.POINTER(nys_options), vp]
        L.nys_update.argtypes = [vp, C.POINTER(nys_instance), vp]
        L.nys_assemble.argtypes = [vp, vp]
        L.nys_solve.argtypes = [vp, vp, vp, vp]
        L.nys_run.argtypes = [vp, vp, vp, vp]
        L.nys_x_stride.argtypes = [vp]
        L.nys_assembly_config.argtypes = [vp, vp, C.POINTER(i32), C.POINTER(i32)]
        L.nys_assembly_items.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.nys_upload_bytes.argtypes = [vp]
        L.nys_upload_bytes.restype = C.c_int64
        L.nys_m_eff.argtypes = [vp, vp, C.POINTER(i32)]
        L.nys_eval.argtypes = [vp, vp, vp, vp, i32, vp]
        L.nys_newton.argtypes = [vp, vp, i32, dbl, vp, vp, vp, vp, vp]
        L.nys_grad.argtypes = [vp, vp, vp, vp, vp, vp]
        L.nys_set_wait_limit.argtypes = [vp, i32]
        L.nys_set_wait_limit.restype = i32
        L.nys_solve_noalloc.argtypes = [C.POINTER(nys_instance), i32, vp, vp, vp]
        L.nys_solve_noalloc.restype = i32
        L.nys_destroy.argtypes = [vp]
        L.nys_destroy.restype = None
        L.nys_status_str.argtypes = [i32]
        L.nys_status_str.restype = C.c_char_p
        L.nys_last_error.argtypes = []
        L.nys_last_error.restype = C.c_char_p
        for name in ("nys_setup", "nys_update", "nys_assemble", "nys_solve", "nys_run",
                     "nys_x_stride", "nys_m_eff", "nys_eval", "nys_newton", "nys_grad",
                     "nys_assembly_config", "nys_assembly_items"):
            getattr(L, name).restype = i32
        _LIB = L
    return _LIB


def check(code):
    if code != NYS_OK:
        raise NysError(code, lib().nys_last_error().decode())
    return code


# ---- the C entry points, same names ------------------------------------------
def nys_setup(inst_array, batch, opt, stream):
    ctx = C.c_void_p()
    check(lib().nys_setup(C.byref(ctx), inst_array, batch, C.byref(opt), stream))
    return ctx


def nys_update(ctx, inst_array, stream):
    check(lib().nys_update(ctx, inst_array, stream))


def nys_assemble(ctx, stream):
    check(lib().nys_assemble(ctx, stream))


def nys_solve(ctx, stream, x_out, status_out):
    check(lib().nys_solve(ctx, stream, x_out, status_out))


def nys_run(ctx, stream, x_out, status_out):
    check(lib().nys_run(ctx, stream, x_out, status_out))


def nys_x_stride(ctx):
    return lib().nys_x_stride(ctx)


def nys_assembly_config(ctx, stream):
    kernel, rows = C.c_int32(), C.c_int32()
    check(lib().nys_assembly_config(ctx, stream, C.byref(kernel), C.byref(rows)))
    return kernel.value, rows.value


def nys_assembly_items(ctx):
    band, other = C.c_int32(), C.c_int32()
    check(lib().nys_assembly_items(ctx, C.byref(band), C.byref(other)))
    return band.value, other.value


def nys_upload_bytes(ctx):
    return lib().nys_upload_bytes(ctx)


def nys_m_eff(ctx, stream, out_array):
    check(lib().nys_m_eff(ctx, stream, out_array))


def nys_eval(ctx, stream, tq, tq_off, deriv, yq_out):
    check(lib().nys_eval(ctx, stream, tq, tq_off, deriv, yq_out))


def nys_newton(ctx, stream, max_iter, tol, warm, x_out, y_aux_out, iters_out, status_out):
    check(lib().nys_newton(ctx, stream, max_iter, tol, warm, x_out, y_aux_out, iters_out, status_out))


def nys_grad(ctx, stream, obs_t, obs_off, dl_dy, grad_out):
    check(lib().nys_grad(ctx, stream, obs_t, obs_off, dl_dy, grad_out))


def nys_set_wait_limit(ctx, polls):
    check(lib().nys_set_wait_limit(ctx, polls))


def nys_solve_noalloc(inst_array, batch, x_out, status_out, stream):
    check(lib().nys_solve_noalloc(inst_array, batch, x_out, status_out, stream))


def nys_destroy(ctx):
    lib().nys_destroy(ctx)


EXPORTS = ("nys_setup", "nys_update", "nys_assemble", "nys_solve", "nys_run", "nys_x_stride",
           "nys_upload_bytes", "nys_assembly_config", "nys_assembly_items",
           "nys_m_eff", "nys_eval", "nys_newton", "nys_grad", "nys_solve_noalloc", "nys_destroy",
           "nys_set_wait_limit",
           "nys_status_str",
           "nys_last_error")
