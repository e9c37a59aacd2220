"""The allocation-free entry point nys_solve_noalloc.

Some callers cannot call cudaMalloc: processes whose device memory is reserved
up front by another allocator (a framework's caching pool, a fixed-budget
server), or latency-critical code that cannot take an allocation's implicit
device synchronisation.  nys_solve_noalloc serves them from one static device
array.  Here it must give the solution of the regular FP64 path (nys_setup +
nys_assemble + nys_solve) on two calls in a row that share that array, and its
fitted y must meet the FP64 bar against the CPU oracle.  This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import nys_inputs as ni
from oracle import core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_04094_gb300 import _abi, api
    return torch, _abi, api


def _problems():
    # m0 at n = 3000 has enough rows for the largest chunk count; one instance sits
    # at the landmark cap NYS_NOALLOC_MAX_M = 64
    return (ni.m0(6, n=3000, m=50) + ni.m0(1, n=2500, m=64) + ni.small_linear(10) + [ni.cfg1()]
            + ni.small_bvp(6, sub=1))


def test_noalloc_matches_regular_fp64_path_and_oracle_twice(env):
    torch, A, api = env
    from parity_helpers import tolerance
    probs = _problems()
    B = len(probs)
    assert max(q["m"] for q in probs) == 64
    ref = api.Batch(probs, precision="fp64")
    ref.assemble()
    xr, sr = ref.solve()
    grids = [core.grid(q) for q in probs]
    yr, _ = ref.eval(grids)
    torch.cuda.synchronize()
    xr = xr.cpu().numpy().copy()
    yr = yr.cpu().numpy()
    assert (sr.cpu().numpy() == 0).all()
    XS = ref.XS
    ref.close()
    # the regular path against the oracle, per instance: err_r and the bar
    err_r, bar, scale = [], [], []
    off = 0
    for q, g in zip(probs, grids):
        tol, sc, o1, _, _ = tolerance(q, g)
        err_r.append(np.abs(yr[off:off + len(g)] - o1["y"]).max() / sc)
        bar.append(tol)
        scale.append(sc)
        off += len(g)
    arr, keep = api.pack_instances(probs)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = torch.full((B, XS), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((B,), 99, dtype=torch.int32, device="cuda")
        A.nys_solve_noalloc(arr, B, C.c_void_p(x.data_ptr()), C.c_void_p(st.data_ptr()), stream)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all(), call
        xn = x.cpu().numpy()
        for b in range(B):
            wr, wn = xr[b, :XS - 2], xn[b, :XS - 2]       # omega (padded), b
            assert np.abs(wn - wr).max() <= 1e-10 * np.abs(wr).max(), (call, b)
            lr, ln = xr[b, XS - 2:], xn[b, XS - 2:]
            assert np.abs(ln - lr).max() <= 1e-7 * max(1.0, np.abs(lr).max()), (call, b)
            # Both paths fit y = omega^T phi(t) + b with the same features phi.
            # phi(t)^T phi(t) = k(t)^T Omega^-1 k(t) <= K(t, t) = 1 (the Nystrom
            # approximation never exceeds the kernel on the diagonal), so for every t
            # |y_noalloc(t) - y_regular(t)| <= |d omega|_2 + |d b|, and the fitted y of
            # this call is within err_r + that bound of the oracle's.
            d = np.linalg.norm(wn[:-1] - wr[:-1]) + abs(wn[-1] - wr[-1])
            assert err_r[b] + d / scale[b] <= bar[b], (call, b, err_r[b], d / scale[b], bar[b])


def test_noalloc_rejects_oversize_requests(env):
    torch, A, api = env
    probs = ni.m0(33, n=500, m=20)
    arr, keep = api.pack_instances(probs)
    x = torch.empty((33, 23), dtype=torch.float64, device="cuda")
    st = torch.empty(33, dtype=torch.int32, device="cuda")
    code = A.lib().nys_solve_noalloc(arr, 33, C.c_void_p(x.data_ptr()), C.c_void_p(st.data_ptr()), None)
    assert code == A.NYS_EINVAL
    assert b"NYS_NOALLOC_MAX_BATCH" in A.lib().nys_last_error()
    big = [dict(ni.cfg1(), m=80, n=400)]
    arr, keep = api.pack_instances(big)
    code = A.lib().nys_solve_noalloc(arr, 1, C.c_void_p(x.data_ptr()), C.c_void_p(st.data_ptr()), None)
    assert code == A.NYS_EINVAL
