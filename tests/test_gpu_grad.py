"""GPU adjoint gradient (nys_grad, NysSolve) against the oracle.

The oracle differentiates the kernel-coordinate form of Lemma 1's problem by
the complex-step method (exact to rounding for this real-analytic map) and, as a
second route, by central differences of the eigen-route solver.  Against the
complex step the bound is 1e-8 of the largest entry of the oracle's gradient
(measured on the gradient workload's family: at most 1.2e-13).  Central
differences carry their own truncation error (about 1e-6 here) and are held to
1e-4.
"""
import numpy as np
import pytest

import nys_inputs as ni
from oracle import adjoint, core

pytestmark = pytest.mark.gpu
RTOL = 1e-8


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_04094_gb300 import api as A
    return A


def _gpu_grad(api, probs, taus, weights):
    """Gradient of l = sum_j w_j y^(tau_j) per instance (upstream = w)."""
    import torch
    bt = api.Batch(probs, precision="fp64")
    bt.assemble()
    x, st = bt.solve()
    g = bt.grad(list(taus), None, np.concatenate(weights))
    y, _ = bt.eval(list(taus))
    torch.cuda.synchronize()
    out = g.cpu().numpy(), y.cpu().numpy(), st.cpu().numpy()
    bt.close()
    return out


def _lin_loss(w):
    return lambda yh, _y: np.sum(w * yh)  # noqa: E731


def _assert_close(got, ref, what):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= RTOL * scale, (what, err / scale, got, ref)


def test_linear_functional_matches_complex_step(api):
    """cfg4's family (p = 2, cos forcing, n = 5000, m = 50, 200 observations)."""
    probs, tau, _ = ni.cfg4(B=3, n_obs=200)
    rng = np.random.default_rng(11)
    w = [rng.standard_normal(len(t)) for t in tau]
    g, _, st = _gpu_grad(api, probs, tau, w)
    assert (st == 0).all()
    for k, q in enumerate(probs):
        ref = adjoint.complex_step_gradient(q, tau[k], None, loss=_lin_loss(w[k]))
        _assert_close(g[k], ref, k)


def test_mse_through_autograd(api):
    """NysSolve: theta -> y^(tau) -> MSE, backward through nys_grad."""
    import torch
    probs, tau, yobs = ni.cfg4(B=2, n=2000, m=40, n_obs=120)
    bt = api.Batch(probs, precision="fp64")
    theta = torch.tensor(api.theta_of(probs), dtype=torch.float64, requires_grad=True)
    tq, tq_off = bt._queries(list(tau), None)
    yhat = api.NysSolve.apply(theta, bt, tq, tq_off)
    yo = torch.tensor(np.concatenate(yobs), dtype=torch.float64, device=yhat.device)
    n_obs = tau.shape[1]
    loss = ((yhat - yo) ** 2).sum() / n_obs   # sum over instances of each instance's MSE
    loss.backward()
    g = theta.grad.cpu().numpy()
    for k, q in enumerate(probs):
        ref = adjoint.complex_step_gradient(q, tau[k], yobs[k])
        _assert_close(g[k], ref, k)
    bt.close()


def test_first_order_and_ragged_batch(api):
    """p = 1 instances (a_2 and y0' entries zero) beside p = 2 ones, ragged n and m,
    ragged observation counts (one instance without observations)."""
    rng = np.random.default_rng(3)
    probs, taus, ws = [], [], []
    for k, (p, n, m, nob) in enumerate([(1, 700, 20, 30), (2, 1500, 32, 50), (1, 333, 13, 0),
                                        (2, 901, 50, 17)]):
        T = float(rng.uniform(4, 12))
        q = dict(p=p, n=n, m=m, t0=0.0, t1=T, sigma=T / m * 1.3, gamma=1e8,
                 v=[float(x) for x in rng.standard_normal(p)], kind="lin",
                 a=[float(rng.uniform(0.2, 1)), float(rng.uniform(1, 3))][:p],
                 c=float(rng.uniform(-1, 1)), omega=float(rng.uniform(0.5, 3)),
                 phi0=float(rng.uniform(0, 3)))
        probs.append(q)
        taus.append(np.sort(rng.uniform(0, T, nob)))
        ws.append(rng.standard_normal(nob))
    g, _, st = _gpu_grad(api, probs, taus, ws)
    assert (st == 0).all()
    for k, q in enumerate(probs):
        if len(taus[k]) == 0:
            assert np.all(g[k] == 0.0)
            continue
        ref = adjoint.complex_step_gradient(q, taus[k], None, loss=_lin_loss(ws[k]))
        _assert_close(g[k], ref, k)
        if q["p"] == 1:
            assert g[k][1] == 0.0 and g[k][5] == 0.0


def test_linearity_identity_full_size(api):
    """At cfg4's full size (1024 instances): the fit is linear in (c, y0, y0'), so
    l = c dl/dc + y0 dl/dy0 + y0' dl/dy0' for a linear functional l = sum w_j y^(tau_j),
    with l computed from the GPU's own fitted values."""
    probs, tau, _ = ni.cfg4()
    rng = np.random.default_rng(7)
    w = [rng.standard_normal(len(t)) for t in tau]
    g, y, st = _gpu_grad(api, probs, tau, w)
    assert (st == 0).all()
    th = api.theta_of(probs)
    nob = tau.shape[1]
    val = np.array([np.sum(w[k] * y[k * nob:(k + 1) * nob]) for k in range(len(probs))])
    recon = th[:, 2] * g[:, 2] + th[:, 4] * g[:, 4] + th[:, 5] * g[:, 5]
    assert np.all(np.abs(recon - val) <= 1e-8 * np.maximum(1.0, np.abs(val))), \
        np.abs(recon - val).max()
    # and a sample of instances against the oracle
    for k in (0, 511, 1023):
        ref = adjoint.complex_step_gradient(probs[k], tau[k], None, loss=_lin_loss(w[k]))
        _assert_close(g[k], ref, k)


def test_truncated_kernel_sigma_is_nan(api):
    """m_eff < m: every entry but sigma matches central differences of the eigen-route
    oracle; sigma is NaN (it would move the discarded eigenvectors)."""
    q = dict(p=2, n=800, m=40, t0=0.0, t1=4.0, sigma=0.6, gamma=1e7, v=[0.3, -0.2], kind="lin",
             a=[0.4, 2.0], c=0.7, omega=1.3, phi0=0.0)
    assert core.setup(q)["W"].shape[0] < q["m"]
    tau = np.linspace(0.1, 3.9, 25)
    yobs = np.sin(tau)
    import torch
    bt = api.Batch([q], precision="fp64")
    bt.assemble()
    bt.solve()
    y, _ = bt.eval([tau])
    u = 2.0 * (y - torch.tensor(yobs, device=y.device)) / len(tau)
    g = bt.grad([tau], None, u).cpu().numpy()[0]
    bt.close()
    assert np.isnan(g[6])
    ref = adjoint.fd_gradient(q, tau, yobs)
    scale = np.abs(ref[:6]).max()
    assert np.abs(g[:6] - ref[:6]).max() <= 1e-4 * scale, (g, ref)


def test_failed_instance_gets_nan(api):
    probs, tau, _ = ni.cfg4(B=3, n=600, m=20, n_obs=10)
    probs[1] = dict(probs[1], c=float("nan"))
    w = [np.ones(len(t)) for t in tau]
    g, _, st = _gpu_grad(api, probs, tau, w)
    assert st[1] == -6
    assert np.isnan(g[1]).all() and np.isfinite(g[0]).all() and np.isfinite(g[2]).all()


def test_grad_refused_for_mixed_context(api):
    from paper_2510_04094_gb300._abi import NysError
    probs, tau, _ = ni.cfg4(B=1, n=600, m=20, n_obs=10)
    bt = api.Batch(probs, precision="mixed")
    bt.assemble()
    bt.solve()
    with pytest.raises(NysError):
        bt.grad([tau[0]], None, np.ones(10))
    bt.close()
