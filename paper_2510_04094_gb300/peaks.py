"""Measured arithmetic peaks of the current GPU (ctypes binding of
include/nys_peak.h): the denominators of the benchmark's roofline fractions.

Each probe launch is timed with CUDA events on the stream it runs on; the loop
count is scaled until a launch takes about `target_ms`, then the best of `reps`
launches is kept (a peak is a burst figure).
"""
import ctypes as C
import os

from . import build as _build

KINDS = {"ffma": 0, "dfma": 1, "tf32_mma": 2, "bf16_mma": 3}
_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.PEAK_LIB_PATH):
            raise RuntimeError("libnys_peak.so is not built; run paper_2510_04094_gb300.build.build()")
        L = C.CDLL(_build.PEAK_LIB_PATH)
        L.nys_peak_launch.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_double)]
        L.nys_peak_launch.restype = C.c_int32
        _LIB = L
    return _LIB


def measure(kind, target_ms=25.0, reps=5):
    """TFLOP/s of probe `kind` (one of KINDS) on the current device and stream."""
    import torch
    stream = torch.cuda.current_stream()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    handle = C.c_void_p(stream.cuda_stream)

    def one(iters):
        fl = C.c_double()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = lib().nys_peak_launch(KINDS[kind], int(iters), handle, C.c_void_p(err.data_ptr()),
                                   C.byref(fl))
        b.record(stream)
        if rc != 0:
            raise RuntimeError("nys_peak_launch(%s) failed: %d" % (kind, rc))
        torch.cuda.synchronize()
        return fl.value, a.elapsed_time(b)

    iters = 64
    fl, ms = one(iters)
    while ms < target_ms / 4 and iters < (1 << 28):
        iters *= 4
        fl, ms = one(iters)
    iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
    best = None
    for _ in range(reps):
        fl, ms = one(iters)
        if best is None or ms < best[1]:
            best = (fl, ms)
    if int(err.item()) != 0:
        raise RuntimeError("peak probe %s: a bounded wait gave up" % kind)
    return {"tflops": best[0] / (best[1] * 1e-3) / 1e12, "ms": best[1], "iters": iters}
