"""GPU Newton (Lemma 2, FP64) against the oracle's Newton iterates.

Same start, same Gauss-Newton fallback rule and stopping rule on both sides:
the iteration counts and statuses must be equal, and for converged instances
the fitted values agree to 1e-10 relative (FP64 tolerance)."""
import numpy as np
import pytest

import nys_inputs as ni
from oracle import core, newton

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


def _duffing(n, m, gamma, T=6.0):
    return dict(p=2, n=n, m=m, t0=0.0, t1=T, sigma=T / m * 1.3, gamma=gamma, v=[0.4, -0.3],
                kind="nl", P=[0.0, 0.7, 0.0, -1.2], delta=0.25, g=0.6, omega=1.1)


def _run(api, probs, max_iter=50, tol=1e-10):
    import torch
    bt = api.Batch(probs, precision="fp64")
    x, st, iters, yaux = bt.newton(max_iter=max_iter, tol=tol, want_y=True)
    grids = [core.grid(q) for q in probs]
    y, _ = bt.eval(grids)
    torch.cuda.synchronize()
    out = (st.cpu().numpy(), iters.cpu().numpy(), y.cpu().numpy(), yaux.cpu().numpy())
    bt.close()
    return out


def _compare(api, probs, max_iter=50, tol=1e-10, ytol=1e-10):
    st, iters, y, yaux = _run(api, probs, max_iter, tol)
    off = offy = 0
    for k, q in enumerate(probs):
        ref = newton.solve(q, tol=tol, max_iter=max_iter)
        n = q["n"]
        assert iters[k] == ref["iters"], (k, iters[k], ref["iters"])
        assert (st[k] == 0) == ref["converged"], (k, st[k])
        if ref["converged"]:
            err = np.abs(y[off:off + n] - ref["y"]).max() / np.abs(ref["y"]).max()
            erry = np.abs(yaux[offy:offy + n - 1] - ref["y_aux"]).max() / np.abs(ref["y_aux"]).max()
            assert err <= ytol and erry <= 10 * ytol, (k, err, erry)
        else:
            assert st[k] == -5
        off += n
        offy += n - 1


def test_tanh_full_size(api):
    _compare(api, [ni.cfg2_tanh()])


def test_small_tanh_and_duffing(api):
    probs = [dict(ni.cfg2_tanh(n=120, m=12), gamma=1e8), _duffing(150, 14, 1e8),
             _duffing(97, 9, 1e6), dict(ni.cfg2_tanh(n=333, m=21), gamma=1e10)]
    _compare(api, probs)


def test_logistic_and_duffing_batch(api):
    """The batched nonlinear family (logistic and Duffing, sigma = T/m), n capped."""
    probs = ni.cfg5(B=8, n_lo=800, n_hi=3000)
    _compare(api, probs, max_iter=20)


def test_cfg5_full_size(api):
    """The batched nonlinear family at its full size: 64 logistic / Duffing instances,
    n in [2000, 1e4], m = 50, cap 20.  The GPU takes the oracle's iteration count and
    status on every instance, and matches its fit on the converged ones.  Under the
    undamped start of the stated reading 18 instances (15 Duffing, 3 logistic) are
    still iterating at the cap on both sides: NYS_ENOCONV, checked here as such."""
    probs = ni.cfg5()
    assert len(probs) == 64 and min(q["n"] for q in probs) >= 2000
    _compare(api, probs, max_iter=20)


def test_linear_rhs_converges_in_one_step(api):
    q = dict(_duffing(200, 12, 1e8), P=[0.3, -1.5, 0.0, 0.0])
    st, iters, y, yaux = _run(api, [q])
    assert st[0] == 0 and iters[0] == 2


def test_iteration_cap_reports_no_convergence(api):
    q = ni.cfg2_tanh(n=500, m=20)
    st, iters, y, yaux = _run(api, [q], max_iter=2)
    assert st[0] == -5 and iters[0] == 2
