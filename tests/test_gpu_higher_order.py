"""GPU parity of orders 3 and 4 (Lemma 1 for general p; Problem 16's fourth-order
boundary value problem, Appendix A.4) against the FP64 oracle, through the C ABI.

FP64 only (the library refuses MIXED for p > 2).  Tolerance: max|y_gpu - y_oracle|
/ max|y_oracle| <= 1e-10, or 10x the spread among the oracle's own exact routes
(LU, null space, and an SVD-computed landmark factor) where the problem itself is
that sensitive."""
import numpy as np
import pytest

import nys_inputs as ni
from oracle import core

from parity_helpers import check_fp64 as _check
from test_oracle_bvp import p16_problem

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


def test_small_ragged_third_and_fourth_order_batch(api):
    """n from 9 to 300, m from 4 to 20, orders 3 and 4, initial and boundary values,
    one batch (several landmark sets, ragged tails)."""
    _check(api, ni.small_higher(16))


def test_orders_1_to_4_in_one_batch(api):
    """Instances of every order share the kernels: the row coefficients and the
    condition rows follow each instance's p."""
    probs = ni.small_higher(6, sub=1) + ni.small_linear(4, p_choices=(1, 2)) + ni.small_bvp(2, sub=2)
    _check(api, probs)


@pytest.mark.parametrize("p,T,m,n,tol", [(3, 3.0, 20, 300, 5e-5), (4, 2.0, 16, 200, 1e-3)])
def test_higher_order_ivps_follow_cos(api, p, T, m, n, tol):
    """y''' + y' = 0 and y'''' = y with the initial values of cos t."""
    t = np.linspace(0.0, T, n)
    z = np.zeros(n)
    f = [z, -np.ones(n), z] if p == 3 else [z, z, z, np.ones(n)]
    q = dict(p=p, n=n, m=m, t0=0.0, t1=T, sigma=1.0, gamma=1e10, v=[1.0, 0.0, -1.0, 0.0][:p],
             kind="table", f=f, r=z)
    (y,) = _check(api, [q])
    assert np.abs(y - np.cos(t)).max() <= tol


def test_problem_16(api):
    """y'''' = 120 t on [-1, 1], y and y' at both ends: parity with the oracle at the
    default eigenvalue cut, and with eigenpairs kept down to 1e-16 lambda_max the
    paper's printed accuracy (errors within [1/10, 2] x the printed ones)."""
    prob, exact, printed = p16_problem()
    _check(api, [prob])
    (y,) = _check(api, [prob], eig_tau=1e-16, tau=1e-16)
    e = np.abs(y - exact)
    for ours, paper in zip((e.mean(), np.sqrt((e ** 2).mean()), e.max()), printed):
        assert paper / 10 <= ours <= 2 * paper, (ours, paper)


def test_higher_orders_refuse_mixed_and_gradients(api):
    import torch
    from paper_2510_04094_gb300 import _abi as A
    with pytest.raises(A.NysError) as e:
        api.Batch(ni.small_higher(2, sub=3), precision="mixed")
    assert e.value.code == A.NYS_EINVAL
    q = [q for q in ni.small_higher(8, sub=4) if q["bc"] == "ivp"][:1]
    bt = api.Batch(q, precision="fp64")
    bt.run()
    torch.cuda.synchronize()
    with pytest.raises(A.NysError) as e:
        bt.grad([np.array([q[0]["t0"] + 0.1])], None, np.ones(1))
    assert e.value.code == A.NYS_EINVAL
    bt.close()
