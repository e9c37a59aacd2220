"""Pins of the oracle's Newton (Lemma 2) and gradient paths.

F against finite differences of the scalar Lagrangian, the Jacobian against
finite differences of F, dense vs y-eliminated steps, one-step convergence for
a linear right-hand side, closed-form solutions, quadratic convergence
(Eq. 3.2.5), a general-purpose constrained minimiser; complex-step gradient vs
finite differences of the eigen route, linearity and zero-residual identities.
"""
import math

import numpy as np
import pytest

import nys_inputs as ni
from oracle import adjoint, core, newton


def _duffing(n=40, m=8, gamma=1e3):
    return dict(p=2, n=n, m=m, t0=0.0, t1=6.0, sigma=6.0 / m * 1.3, gamma=gamma, v=[0.4, -0.3],
                kind="nl", P=[0.0, 0.7, 0.0, -1.2], delta=0.25, g=0.6, omega=1.1)


def _tanh(n=40, m=8, gamma=1e3):
    return dict(ni.cfg2_tanh(n=n, m=m), gamma=gamma)


@pytest.mark.parametrize("mk", [_tanh, _duffing])
def test_F_is_gradient_of_lagrangian(mk):
    pc = newton.Pieces(mk())
    rng = np.random.default_rng(1)
    x = newton.x0(pc) + 0.3 * rng.standard_normal(pc.me + 1 + pc.p + pc.n1)
    F = pc.F(x)
    h = 1e-6
    fd = np.array([(pc.lagrangian(x + h * e) - pc.lagrangian(x - h * e)) / (2 * h)
                   for e in np.eye(len(x))])
    assert np.abs(F - fd).max() <= 1e-6 * np.abs(F).max()


@pytest.mark.parametrize("mk", [_tanh, _duffing])
def test_jacobian_is_derivative_of_F(mk):
    pc = newton.Pieces(mk())
    rng = np.random.default_rng(2)
    x = newton.x0(pc) + 0.3 * rng.standard_normal(pc.me + 1 + pc.p + pc.n1)
    J = pc.J(x)
    h = 1e-6
    fd = np.array([(pc.F(x + h * e) - pc.F(x - h * e)) / (2 * h) for e in np.eye(len(x))]).T
    assert np.abs(J - fd).max() <= 1e-6 * np.abs(J).max()
    # Gauss-Newton differs only on the y-diagonal, by gamma * e_i * P''(y_i)
    Jg = pc.J(x, gauss_newton=True)
    e, xi, hh, Q, f_y, f_yy, f_yu, f_uu = pc.residuals(x)
    D = J - Jg
    oy = pc.me + 1 + pc.p
    np.testing.assert_allclose(np.diag(D)[oy:], -pc.gamma * e * f_yy, rtol=1e-12, atol=1e-9)
    D[oy + np.arange(pc.n1), oy + np.arange(pc.n1)] = 0
    assert np.abs(D).max() == 0


@pytest.mark.parametrize("mk", [_tanh, _duffing])
def test_dense_and_reduced_newton_agree(mk):
    prob = mk(n=120, m=12, gamma=1e8)
    a = newton.solve(prob, dense=True, history=True)
    b = newton.solve(prob, dense=False, history=True)
    assert a["iters"] == b["iters"] and a["converged"] and b["converged"]
    pc = a["pieces"]
    for ha, hb in zip(a["history"], b["history"]):
        # (omega, b, y) to 1e-8; the multipliers of an early iterate are less well
        # determined (rounding of the two elimination orders) and get 1e-6
        for blk_a, blk_b, tol in zip(pc.split(ha["x"]), pc.split(hb["x"]), (1e-8, 1e-8, 1e-6, 1e-8)):
            blk_a, blk_b = np.atleast_1d(blk_a), np.atleast_1d(blk_b)
            assert np.abs(blk_a - blk_b).max() <= tol * max(1.0, np.abs(blk_a).max())
    assert np.abs(a["y"] - b["y"]).max() <= 1e-10 * np.abs(a["y"]).max()


def test_linear_right_hand_side_converges_in_one_step():
    """With P linear in y the Lagrangian is quadratic: one Newton step solves F = 0."""
    prob = dict(_duffing(n=80, m=10, gamma=1e6), P=[0.3, -1.5, 0.0, 0.0])
    sol = newton.solve(prob, history=True)
    pc = sol["pieces"]
    F1 = pc.F(sol["history"][1]["x"])
    F0 = pc.F(sol["history"][0]["x"])
    assert np.linalg.norm(F1) <= 1e-9 * np.linalg.norm(F0)
    assert sol["iters"] == 2 and sol["converged"]


def test_linear_rhs_nonlinear_form_matches_lemma1():
    """y' = c0 + c1 y through Lemma 2 and through Lemma 1: with gamma = 1e10 the
    auxiliary penalty pins y_i to the model, and the two fits coincide."""
    nl = dict(p=1, n=300, m=20, t0=0.0, t1=3.0, sigma=0.5, gamma=1e10, v=[0.5], kind="nl",
              P=[0.2, -0.8, 0.0, 0.0], delta=0.0, g=0.0, omega=0.0)
    lin = dict(p=1, n=300, m=20, t0=0.0, t1=3.0, sigma=0.5, gamma=1e10, v=[0.5], kind="lin",
               a=[0.8], c=0.2, omega=0.0, phi0=math.pi / 2)
    a = newton.solve(nl)
    b = core.solve_linear(lin)
    exact = 0.25 + 0.25 * np.exp(-0.8 * a["t"])
    assert np.abs(a["y"] - b["y"]).max() < 1e-9
    assert np.abs(a["y"] - exact).max() < 2e-5 and np.abs(b["y"] - exact).max() < 2e-5


def test_newton_solution_is_a_kkt_point_and_converges_quadratically():
    prob = ni.cfg2_tanh(n=2000, m=30)
    sol = newton.solve(prob, history=True)
    assert sol["converged"] and sol["iters"] <= 20
    pc = sol["pieces"]
    hist = sol["history"]
    steps = [np.linalg.norm(hist[k + 1]["x"] - hist[k]["x"]) for k in range(len(hist) - 1)]
    # Eq. 3.2.5: in the quadratic phase |d_{k+1}| <= K |d_k|^2 with a moderate K
    ratios = [steps[k + 1] / steps[k] ** 2 for k in range(len(steps) - 1)
              if 1e-9 < steps[k] < 1e-1 and steps[k + 1] > 1e-12]
    assert ratios and max(ratios) < 1e3
    F0 = np.linalg.norm(pc.F(hist[0]["x"]))
    assert np.linalg.norm(pc.F(hist[-1]["x"])) <= 1e-10 * F0


def test_tanh_and_logistic_closed_forms():
    sol = newton.solve(ni.cfg2_tanh(n=4000, m=50))
    assert sol["converged"]
    assert np.abs(sol["y"] - np.tanh(sol["t"])).max() < 1e-5
    # logistic y' = r y (1 - y/K); from the default start (y_i = y(0)) Newton reaches the
    # true branch when y(0)/K is not small (for y(0) << K it can settle on y = 0)
    for (r, K, y0, T) in ((1.0, 2.0, 1.0, 8.0), (0.8, 3.0, 1.0, 10.0)):
        prob = dict(p=1, n=3000, m=50, t0=0.0, t1=T, sigma=T / 25, gamma=1e10, v=[y0], kind="nl",
                    P=[0.0, r, -r / K, 0.0], delta=0.0, g=0.0, omega=0.0, logistic=(r, K, y0))
        sol = newton.solve(prob, max_iter=30)
        assert sol["converged"]
        assert np.abs(sol["y"] - ni.closed_form_logistic(prob, sol["t"])).max() < 5e-3 * K


def test_newton_point_matches_general_constrained_minimiser():
    """scipy SLSQP on the objective of Eq. 2.2 written from its definition."""
    from scipy.optimize import minimize
    prob = _tanh(n=15, m=5, gamma=5.0)
    sol = newton.solve(prob)
    pc = sol["pieces"]
    me, p = pc.me, pc.p

    def obj(z):
        x = np.concatenate([z[:me + 1], np.zeros(p), z[me + 1:]])
        om, b, lam, y = pc.split(x)
        e, xi, h, *_ = pc.residuals(x)
        return 0.5 * om @ om + 0.5 * pc.gamma * (e @ e + xi @ xi)

    def cons(z):
        x = np.concatenate([z[:me + 1], np.zeros(p), z[me + 1:]])
        return pc.residuals(x)[2]

    xs = np.concatenate([sol["omega"], [sol["b"]], sol["y_aux"]])
    res = minimize(obj, xs + 0.05, constraints=[dict(type="eq", fun=cons)], method="SLSQP",
                   options=dict(ftol=1e-14, maxiter=500))
    assert res.success
    assert np.abs(res.x - xs).max() < 1e-5 * max(1, np.abs(xs).max())


# --------------------------------------------------------------- gradient ----
def _grad_problem(n=600, m=30):
    prob = ni.cfg4(B=1, n=n, m=m, n_obs=40)
    return prob[0][0], prob[1][0], prob[2][0]


def test_complex_step_gradient_matches_finite_differences():
    prob, tau, yobs = _grad_problem()
    gc = adjoint.complex_step_gradient(prob, tau, yobs)
    gf = adjoint.fd_gradient(prob, tau, yobs)
    assert np.abs(gc - gf).max() <= 1e-5 * np.abs(gc).max()


def test_gradient_linearity_identity():
    """The fit is linear in (c, y0, y0'): for l = sum_j w_j y^(tau_j),
    l = c dl/dc + y0 dl/dy0 + y0' dl/dy0'."""
    prob, tau, _ = _grad_problem(n=400)
    w = np.random.default_rng(5).standard_normal(len(tau))
    loss = lambda yh, _y: np.sum(w * yh)  # noqa: E731
    g = adjoint.complex_step_gradient(prob, tau, None, loss=loss)
    val = np.sum(w * adjoint.fitted(prob, tau).real)
    th = adjoint._unpack(prob)
    recon = th["c"] * g[2] + th["y0"] * g[4] + th["y0p"] * g[5]
    assert abs(recon - val) <= 1e-9 * max(1, abs(val))


def test_gradient_vanishes_at_exact_fit():
    prob, tau, yobs = _grad_problem(n=400)
    yfit = adjoint.fitted(prob, tau).real
    g = adjoint.complex_step_gradient(prob, tau, yfit)
    g_noisy = adjoint.complex_step_gradient(prob, tau, yobs)
    assert np.abs(g).max() < 1e-10 * np.abs(g_noisy).max()


def _problem15(n=60, m=10, gamma=1e4):
    """Appendix A.6: y'' = -y + 2 (y')^2 / y on [-1, 1], y(-1) = y(1) = 0.324027137."""
    q = 0.5 / np.cosh(1.0)
    return dict(p=2, n=n, m=m, t0=-1.0, t1=1.0, sigma=1.0, gamma=gamma, v=[q, q], kind="nl",
                P=[0.0, -1.0, 0.0, 0.0], delta=0.0, beta=2.0, g=0.0, omega=0.0, bc="bvp")


def test_jacobian_is_derivative_of_F_with_nonlinear_derivative_term():
    """f nonlinear in u = y' (the u^2 / y term of Problem 15): the per-row
    d e / d omega and the - e f_uu phi' phi'^T and - e f_yu phi' Hessian terms,
    against central differences of F."""
    pc = newton.Pieces(_problem15())
    rng = np.random.default_rng(3)
    x = newton.x0(pc) + 0.05 * rng.standard_normal(pc.me + 1 + pc.p + pc.n1)
    x[pc.me + 1 + pc.p:] = np.abs(x[pc.me + 1 + pc.p:]) + 0.2     # y_i away from 0
    J = pc.J(x)
    h = 1e-6
    fd = np.array([(pc.F(x + h * e) - pc.F(x - h * e)) / (2 * h) for e in np.eye(len(x))]).T
    assert np.abs(J - fd).max() <= 1e-6 * np.abs(J).max()
    # the reduced (y-eliminated) step equals the dense one
    a = newton.step_dense(pc, x, False)
    b = newton.step_reduced(pc, x, False)
    assert np.abs(a - b).max() <= 1e-8 * max(1.0, np.abs(a).max())


def test_duffing_matches_an_independent_integrator():
    """The Duffing equation y'' = 0.7 y - 1.2 y^3 - 0.25 y' + 0.6 cos(1.1 t) on [0, 6],
    y(0) = 0.4, y'(0) = -0.3, has no closed form.  The oracle's Newton fit (Lemma 2)
    is compared with an explicit Runge-Kutta integration of order 8 (scipy's DOP853,
    tolerances 1e-13), an independent method.  Measured: 1.0e-6 relative at n = 2000,
    m = 50, sigma = 1 and 5.2e-7 at n = 4000, m = 100.  That is the method's
    discretisation error, shrinking with resolution.  A wrong sign of the damping, the
    linear, the cubic or the forcing term, or of y'(0), moves the error to 0.8 or more
    (or the integration blows up)."""
    integrate = pytest.importorskip("scipy.integrate")

    def rhs(t, s):
        y, u = s
        return [u, 0.7 * y - 1.2 * y ** 3 - 0.25 * u + 0.6 * math.cos(1.1 * t)]

    errs = []
    for n, m in ((2000, 50), (4000, 100)):
        prob = dict(p=2, n=n, m=m, t0=0.0, t1=6.0, sigma=1.0, gamma=1e10, v=[0.4, -0.3],
                    kind="nl", P=[0.0, 0.7, 0.0, -1.2], delta=0.25, g=0.6, omega=1.1)
        sol = newton.solve(prob)
        assert sol["converged"]
        t = core.grid(prob)
        ref = integrate.solve_ivp(rhs, [0.0, 6.0], [0.4, -0.3], method="DOP853", rtol=1e-13,
                                  atol=1e-13, t_eval=t)
        assert ref.success and ref.y.shape[1] == len(t)
        errs.append(np.abs(sol["y"] - ref.y[0]).max() / np.abs(ref.y[0]).max())
    assert errs[0] <= 5e-6, errs
    assert errs[1] <= 2e-6 and errs[1] < errs[0], errs
