"""Thin PyTorch-facing wrapper over the C ABI (argument marshalling only).

PyTorch provides device memory (torch tensors) and the CUDA stream; every
computation happens in libnys.so.  Problems are plain dicts (see
``nys_inputs``): p, n, m, t0, t1, sigma, gamma, v, kind, the kind-specific
coefficients and optionally bc ('ivp', the default, or 'bvp').
"""
import ctypes as C

import numpy as np
import torch

from . import _abi as A

_KIND = {"table": A.NYS_COEF_TABLE, "lin": A.NYS_COEF_LIN, "nl": A.NYS_COEF_POLY_NL}
_BC = {"ivp": A.NYS_BC_IVP, "bvp": A.NYS_BC_BVP}

# order of the gradient entries of nys_grad (kind "lin")
THETA = ("a", "b", "c", "omega", "y0", "y0p", "sigma")


def _stream_handle(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def pack_instances(problems):
    """Marshal problem dicts into a ctypes nys_instance array (+ keep-alive buffers)."""
    B = len(problems)
    arr = (A.nys_instance * B)()
    keep = []
    for b, q in enumerate(problems):
        s = arr[b]
        s.p, s.n, s.m = int(q["p"]), int(q["n"]), int(q["m"])
        s.kind = _KIND[q["kind"]]
        s.bc = _BC[q.get("bc", "ivp")]
        s.t0, s.t1 = float(q["t0"]), float(q["t1"])
        s.sigma, s.gamma = float(q["sigma"]), float(q["gamma"])
        v = list(q["v"]) + [0.0] * (4 - len(q["v"]))
        for k in range(4):
            s.v[k] = float(v[k])
        c = [0.0] * 8
        if q["kind"] == "lin":
            a = list(q["a"]) + [0.0] * (2 - len(q["a"]))
            c[0], c[1] = a[0], a[1]
            c[2], c[3], c[4] = q["c"], q["omega"], q.get("phi0", 0.0)
        elif q["kind"] == "nl":
            c[0:4] = list(q["P"])
            c[4], c[5], c[6] = q.get("delta", 0.0), q.get("g", 0.0), q.get("omega", 0.0)
            c[7] = q.get("beta", 0.0)
        elif q["kind"] == "table":
            tabv = np.ascontiguousarray(np.concatenate(
                [np.asarray(q["f"], dtype=np.float64).reshape(s.p, s.n),
                 np.asarray(q["r"], dtype=np.float64).reshape(1, s.n)]), dtype=np.float64)
            keep.append(tabv)
            s.coef_table = tabv.ctypes.data_as(C.POINTER(C.c_double))
        for k in range(8):
            s.c[k] = float(c[k])
        if q.get("landmarks") is not None:
            lmv = np.ascontiguousarray(q["landmarks"], dtype=np.int32)
            keep.append(lmv)
            s.landmarks = lmv.ctypes.data_as(C.POINTER(C.c_int32))
    return arr, keep


class Batch:
    """A batch of ODE instances bound to one nys_ctx on the current CUDA device."""

    def __init__(self, problems, precision="fp64", refine_steps=-1, eig_tau=0.0,
                 scale_sqrt_m=False, stream=None, assembly="auto"):
        """precision: "fp64", "mixed" or "mixed-f64f" (nys_precision); assembly (mixed
        precisions): "auto", "tc", "simt" or "tune" (nys_assembly).  refine_steps
        (mixed): residual passes for every instance; negative selects the default,
        one pass (two with boundary values) and then an adaptive pass for the
        instances whose estimated error is still above 1e-8."""
        self.problems = list(problems)
        self.B = len(self.problems)
        self.stream = stream
        opt = A.nys_options()
        opt.precision = {"fp64": A.NYS_FP64, "mixed": A.NYS_MIXED,
                         "mixed-f64f": A.NYS_MIXED_F64F}[precision]
        opt.refine_steps = int(refine_steps)
        opt.eig_tau = float(eig_tau)
        opt.scale_sqrt_m = 1 if scale_sqrt_m else 0
        opt.assembly = {"auto": A.NYS_ASM_AUTO, "simt": A.NYS_ASM_SIMT, "tune": A.NYS_ASM_TUNE,
                        "tc": A.NYS_ASM_TC}[assembly]
        arr, keep = pack_instances(self.problems)
        self.ctx = A.nys_setup(arr, self.B, opt, _stream_handle(stream))
        self.XS = A.nys_x_stride(self.ctx)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.x = torch.zeros(self.B, self.XS, dtype=torch.float64, device=dev)
        self.status = torch.zeros(self.B, dtype=torch.int32, device=dev)
        self.version = 0   # bumped by every solve; nys_grad differentiates the latest

    def close(self):
        if getattr(self, "ctx", None) is not None:
            A.nys_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, problems):
        arr, keep = pack_instances(problems)
        self.problems = list(problems)
        A.nys_update(self.ctx, arr, _stream_handle(self.stream))

    def assemble(self):
        A.nys_assemble(self.ctx, _stream_handle(self.stream))

    def solve(self):
        A.nys_solve(self.ctx, _stream_handle(self.stream), _ptr(self.x), _ptr(self.status))
        self.version += 1
        return self.x, self.status

    def run(self):
        A.nys_run(self.ctx, _stream_handle(self.stream), _ptr(self.x), _ptr(self.status))
        self.version += 1
        return self.x, self.status

    def assembly_config(self):
        """(kernel, rows per work item) of the assembly; runs the tuner if pending.
        kernel: "auto" (band units on the CUDA cores, the rest on the tensor
        cores), "tensor-core" or "simt"."""
        kernel, rows = A.nys_assembly_config(self.ctx, _stream_handle(self.stream))
        return {A.NYS_ASM_AUTO: "auto", A.NYS_ASM_TC: "tensor-core", A.NYS_ASM_SIMT: "simt"}[kernel], rows

    def assembly_items(self):
        """(band units, other work items) of the assembly work list in use."""
        return A.nys_assembly_items(self.ctx)

    def m_eff(self):
        out = (C.c_int32 * self.B)()
        A.nys_m_eff(self.ctx, _stream_handle(self.stream), out)
        return np.frombuffer(out, dtype=np.int32).copy()

    def eval(self, tq, tq_off=None, deriv=0):
        """tq: list of per-instance query arrays (instances 0..len(tq)-1; the rest get
        none), or a flat CUDA tensor with int64 offsets of length batch + 1."""
        tq, tq_off = self._queries(tq, tq_off)
        y = torch.empty_like(tq)
        A.nys_eval(self.ctx, _stream_handle(self.stream), _ptr(tq), _ptr(tq_off), int(deriv), _ptr(y))
        return y, tq_off

    def _queries(self, tq, tq_off):
        dev = self.x.device
        if tq_off is None:
            if len(tq) > self.B:
                raise ValueError("more query lists than instances")
            lens = [len(a) for a in tq] + [0] * (self.B - len(tq))
            tq_off = torch.tensor(np.r_[0, np.cumsum(lens)], dtype=torch.int64, device=dev)
            tq = torch.tensor(np.concatenate([np.asarray(a, dtype=np.float64) for a in tq]),
                              dtype=torch.float64, device=dev)
        if tq_off.numel() != self.B + 1:
            raise ValueError("tq_off must have batch + 1 entries")
        return tq, tq_off

    def newton(self, max_iter=50, tol=1e-10, want_y=False, warm=None):
        """Newton's method (nys_newton).  warm: optional start (x, y_aux): x in
        x's layout (batch x XS), y_aux the auxiliary unknowns (sum(n - 1)), e.g.
        copies of an earlier call's outputs."""
        dev = self.x.device
        if not hasattr(self, "_nt_iters"):
            # output buffers kept per Batch: nys_newton replays its captured graph
            # for the same pointers
            self._nt_iters = torch.zeros(self.B, dtype=torch.int32, device=dev)
            self._nt_y = torch.empty(sum(q["n"] - 1 for q in self.problems), dtype=torch.float64,
                                     device=dev)
        if warm is not None:
            wx = torch.as_tensor(warm[0], dtype=torch.float64, device=dev).reshape(-1)
            wy = torch.as_tensor(warm[1], dtype=torch.float64, device=dev).reshape(-1)
            ny = self._nt_y.numel()
            if wx.numel() != self.B * self.XS or wy.numel() != ny:
                raise ValueError("warm must be (x: batch x XS, y_aux: sum(n - 1))")
            if not hasattr(self, "_nt_warm"):
                self._nt_warm = torch.empty(self.B * self.XS + ny, dtype=torch.float64, device=dev)
            self._nt_warm[:self.B * self.XS].copy_(wx)
            self._nt_warm[self.B * self.XS:].copy_(wy)
            warm = self._nt_warm
        yaux = self._nt_y if want_y else None
        A.nys_newton(self.ctx, _stream_handle(self.stream), int(max_iter), float(tol), _ptr(warm),
                     _ptr(self.x), _ptr(yaux), _ptr(self._nt_iters), _ptr(self.status))
        return self.x, self.status, self._nt_iters, yaux

    def grad(self, obs_t, obs_off, dl_dy):
        """d loss / d theta (batch x 7, order THETA) of the last solve, given the
        upstream d loss / d y^(obs_t) (flat CUDA float64 tensors as for eval)."""
        obs_t, obs_off = self._queries(obs_t, obs_off)
        dl_dy = torch.as_tensor(dl_dy, dtype=torch.float64, device=self.x.device).contiguous()
        if dl_dy.numel() != obs_t.numel():
            raise ValueError("dl_dy must have one entry per observation time")
        g = torch.empty(self.B, 7, dtype=torch.float64, device=self.x.device)
        A.nys_grad(self.ctx, _stream_handle(self.stream), _ptr(obs_t), _ptr(obs_off), _ptr(dl_dy), _ptr(g))
        return g

    # unpack helpers ---------------------------------------------------------
    def unpack(self):
        x = self.x.cpu().numpy()
        out = []
        for b in range(self.B):
            out.append(dict(omega=x[b, :self.XS - 3], b=x[b, self.XS - 3], lam=x[b, self.XS - 2:]))
        return out


def problems_with_theta(problems, theta):
    """Copies of the "lin" problem dicts with (a_1, a_2, c, omega, y0, y0', sigma)
    taken from the rows of theta (batch x 7)."""
    th = np.asarray(theta, dtype=np.float64).reshape(len(problems), 7)
    out = []
    for q, t in zip(problems, th):
        if q["kind"] != "lin":
            raise ValueError("theta applies to kind 'lin' problems only")
        p = int(q["p"])
        r = dict(q)
        r["a"] = [float(t[0]), float(t[1])][:p]
        r["c"], r["omega"] = float(t[2]), float(t[3])
        r["v"] = [float(t[4]), float(t[5])][:p]
        r["sigma"] = float(t[6])
        out.append(r)
    return out


def theta_of(problems):
    """The batch x 7 parameter array (order THETA) of "lin" problem dicts."""
    th = np.zeros((len(problems), 7))
    for k, q in enumerate(problems):
        a = list(q["a"]) + [0.0] * (2 - len(q["a"]))
        v = list(q["v"]) + [0.0] * (2 - len(q["v"]))
        th[k] = [a[0], a[1], q["c"], q["omega"], v[0], v[1], q["sigma"]]
    return th


class NysSolve(torch.autograd.Function):
    """Fitted values y^(tau) of the FP64 linear solve as a differentiable function of
    theta (batch x 7 float64, order THETA).

    forward: nys_update with theta, nys_assemble, nys_solve, nys_eval at tau.
    backward: nys_grad with the upstream gradient (one adjoint solve + one row pass).
    The Batch must be FP64; backward refers to the Batch's latest solve, so only
    one forward per Batch may be awaiting its backward.
    """

    @staticmethod
    def forward(ctx, theta, batch, tq, tq_off):
        batch.update(problems_with_theta(batch.problems, theta.detach().cpu().numpy()))
        batch.assemble()
        batch.solve()
        y, _ = batch.eval(tq, tq_off)
        ctx.batch, ctx.version, ctx.theta_device = batch, batch.version, theta.device
        ctx.save_for_backward(tq, tq_off)
        return y

    @staticmethod
    def backward(ctx, gy):
        if ctx.batch.version != ctx.version:
            raise RuntimeError("NysSolve: the Batch was solved again after this forward")
        tq, tq_off = ctx.saved_tensors
        g = ctx.batch.grad(tq, tq_off, gy.to(torch.float64).contiguous())
        return g.to(ctx.theta_device), None, None, None
