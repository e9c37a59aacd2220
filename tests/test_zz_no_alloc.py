"""The allocation-free entry point nys_solve_noalloc (for callers that cannot
call cudaMalloc, e.g. processes whose device memory is reserved up front by
another allocator) must give the same solution as the regular FP64 path
(nys_setup + nys_assemble + nys_solve), on two calls in a row that share its
static device workspace.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import nys_inputs as ni

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
    return ni.m0(6, n=3000, m=50) + ni.small_linear(10) + [ni.cfg1()] + ni.small_bvp(6, sub=1)


def test_noalloc_matches_regular_fp64_path_twice(env):
    torch, A, api = env
    probs = _problems()
    B = len(probs)
    ref = api.Batch(probs, precision="fp64")
    ref.assemble()
    xr, sr = ref.solve()
    torch.cuda.synchronize()
    xr = xr.cpu().numpy().copy()
    assert (sr.cpu().numpy() == 0).all()
    XS = ref.XS
    ref.close()
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
            wb_r = np.r_[xr[b, :XS - 2]]
            wb_n = np.r_[xn[b, :XS - 2]]
            scale = np.abs(wb_r).max()
            assert np.abs(wb_n - wb_r).max() <= 1e-10 * scale, (call, b)
            lr, ln = xr[b, XS - 2:], xn[b, XS - 2:]
            assert np.abs(ln - lr).max() <= 1e-7 * max(1.0, np.abs(lr).max()), (call, b)


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
