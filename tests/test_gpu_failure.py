"""Failure paths of the device code, exercised without a GPU fault.

The tensor-core assembly (NYS_ASM_TC here, so that every instance runs on it)
bounds every mbarrier wait (nys_set_wait_limit).  With
the limit at 0 every wait gives up at once: the kernel records its error word,
drains, frees its tensor memory and returns, the solve reports NYS_ETIMEOUT for
every instance, and the same context then solves normally once the default limit
is back -- through the stepwise calls and through a freshly captured nys_run
graph.
"""
import numpy as np
import pytest

import nys_inputs as ni
from oracle import core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_04094_gb300 import api as A
    return A


def _errs(bt, probs):
    import torch
    grids = [core.grid(q) for q in probs]
    y, _ = bt.eval(grids)
    torch.cuda.synchronize()
    yc = y.cpu().numpy()
    off, out = 0, []
    for q, g in zip(probs, grids):
        ref = core.solve_linear(q)["y"]
        out.append(np.abs(yc[off:off + len(g)] - ref).max() / np.abs(ref).max())
        off += len(g)
    return out


def test_expired_waits_report_timeout_and_context_recovers(api):
    import torch
    from paper_2510_04094_gb300 import _abi as A
    probs = ni.m0(6, n=2000, m=30) + ni.small_linear(4, sub=5)
    bt = api.Batch(probs, precision="mixed", assembly="tc")
    A.nys_set_wait_limit(bt.ctx, 0)
    for step in (lambda: (bt.assemble(), bt.solve())[1], bt.run):
        st = step()[1]
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == A.NYS_ETIMEOUT).all()
    A.nys_set_wait_limit(bt.ctx, -1)
    bt.assemble()
    _, st = bt.solve()
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert max(_errs(bt, probs)) <= 1e-6
    _, st = bt.run()
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert max(_errs(bt, probs)) <= 1e-6
    bt.close()


def test_wait_limit_needs_a_context(api):
    from paper_2510_04094_gb300 import _abi as A
    assert A.lib().nys_set_wait_limit(None, 5) == A.NYS_EINVAL
