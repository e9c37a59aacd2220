"""Pins of the oracle's boundary value case (Appendix A.4, BVP: y(t_1) = q_1,
y(t_n) = q_n, collocation rows 2..n-1)."""
import os

import numpy as np
import pytest

from oracle import core

from bvp_problems import golden_rows as _golden_rows
from bvp_problems import problem as _problem


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_paper_bvp_table_accuracy(row):
    """The printed NLS-SVM errors of Problems 11-13 are met.  The paper does not
    state how it treats the numerically singular landmark kernel (20 landmarks,
    sigma = 1 on [0, 1]); keeping eigenpairs down to 1e-16 lambda_max (11 of 20)
    reproduces its figures for P11 and P12 (ours within [1/10, 2] x printed); for
    P13 ours is ~17x more accurate than printed, so only the upper bound applies."""
    name, q1, qn, n, m, s2, gam, mae, rmse, linf = row
    prob, exact = _problem(name, q1, qn, n, m, s2, gam)
    sol = core.solve_linear(prob, tau=1e-16)
    e = np.abs(sol["y"] - exact)
    for ours, paper in ((e.mean(), mae), (np.sqrt((e ** 2).mean()), rmse), (e.max(), linf)):
        assert ours <= 2 * paper, (name, ours, paper)
        if name != "P13":
            assert ours >= paper / 10, (name, ours, paper)


@pytest.mark.parametrize("name", ["P11", "P12", "P13"])
def test_bvp_conditions_met_and_exact_routes_agree(name):
    prob, _ = _problem(*[r for r in _golden_rows() if r[0] == name][0][:7])
    a = core.solve_linear(prob)
    b = core.solve_linear_nullspace(prob)
    # y(t_1) = q_1 and y(t_n) = q_n hold to rounding (the grid evaluation sums
    # large feature weights, so it is looser)
    assert np.max(np.abs(core.constraints(prob, a, a["omega"], a["b"]))) <= 1e-12
    y = a["y"]
    assert abs(y[0] - prob["v"][0]) <= 1e-10 and abs(y[-1] - prob["v"][1]) <= 1e-10
    assert np.max(np.abs(a["y"] - b["y"])) <= 1e-9 * np.max(np.abs(a["y"]))
    # the multipliers carry the conditioning of the KKT matrix (~gamma n): two exact
    # FP64 routes agree to ~1e-4 relative here
    np.testing.assert_allclose(a["lam"], b["lam"], rtol=1e-3)


def _rbf_rows(t, s, sigma):
    """k, k', k'' of exp(-(t - s)^2 / sigma^2) in t, written out for this test."""
    d = t[:, None] - s[None, :]
    k = np.exp(-(d / sigma) ** 2)
    return k, -2 * d / sigma ** 2 * k, (4 * d ** 2 / sigma ** 4 - 2 / sigma ** 2) * k


@pytest.mark.parametrize("seed", [0, 1])
def test_bvp_solution_is_stationary_on_interior_rows_only(seed):
    """First-order optimality of Appendix A.4's problem rebuilt from its statement:
    the gradient of 1/2|w|^2 + gamma/2 sum_{i=2}^{n-1} e_i^2 lies in the span of the
    two condition rows.  Including row n (or row 1) in the sum breaks it."""
    g = np.random.default_rng(seed)
    n, m = 60, 12
    t = np.linspace(0.0, 2.0, n)
    f1, f2 = g.uniform(-1, 1, n), g.uniform(-2, 0, n)
    r = np.sin(3 * t) + g.uniform(-0.1, 0.1, n)
    prob = dict(p=2, n=n, m=m, t0=0.0, t1=2.0, sigma=0.4, gamma=1e4, v=[0.3, -0.7],
                kind="table", f=[f1, f2], r=r, bc="bvp")
    sol = core.solve_linear(prob)
    W, s, me = sol["W"], sol["s"], sol["m_eff"]
    k0, k1, k2 = _rbf_rows(t, s, prob["sigma"])
    P0, P1, P2 = k0 @ W.T, k1 @ W.T, k2 @ W.T
    x = np.concatenate([sol["omega"], [sol["b"]]])

    def grad(rows):
        gr = np.zeros(me + 1)
        gr[:me] = sol["omega"]
        for i in rows:
            a = np.concatenate([P2[i] - f1[i] * P1[i] - f2[i] * P0[i], [-f2[i]]])
            e = a @ x - r[i]
            gr += prob["gamma"] * e * a
        return gr

    C = np.vstack([np.concatenate([P0[0], [1.0]]), np.concatenate([P0[-1], [1.0]])])
    Q, _ = np.linalg.qr(C.T, mode="complete")
    Z = Q[:, 2:]
    good = Z.T @ grad(range(1, n - 1))
    scale = np.abs(prob["gamma"] * P2).max() * 1e-8 + 1e-8
    assert np.max(np.abs(good)) <= scale
    for bad_rows in (range(1, n), range(0, n - 1)):
        assert np.max(np.abs(Z.T @ grad(bad_rows))) > 100 * scale


# ---- nonlinear boundary value problems (Newton, Lemma 2 with the conditions of
# Appendix A.4) ----------------------------------------------------------------
NL_BVP = [
    # y'' = 2 y^3, y(0) = 1, y(1) = 1/2: y = 1/(1+t)
    ("cubic", [0.0, 0.0, 0.0, 2.0], (1.0, 0.5), lambda t: 1 / (1 + t), 1e-6),
    # y'' = y^2, y(0) = 6, y(1) = 3/2: y = 6/(1+t)^2
    ("square", [0.0, 0.0, 1.0, 0.0], (6.0, 1.5), lambda t: 6 / (1 + t) ** 2, 2e-5),
]


def nl_bvp_problem(P, q, n=200, m=20, sigma=0.3, gamma=1e10):
    return dict(p=2, n=n, m=m, t0=0.0, t1=1.0, sigma=sigma, gamma=gamma, v=list(q), kind="nl",
                P=list(P), delta=0.0, g=0.0, omega=0.0, bc="bvp")


@pytest.mark.parametrize("case", NL_BVP, ids=lambda c: c[0])
def test_nonlinear_bvp_matches_closed_form(case):
    """Newton on Lemma 2's Lagrangian with boundary conditions reaches the closed-form
    solution of a polynomial nonlinear BVP; dense and y-eliminated steps agree."""
    from oracle import newton
    name, P, q, exact, tol = case
    prob = nl_bvp_problem(P, q)
    dense = newton.solve(prob, dense=True)
    red = newton.solve(prob, dense=False)
    assert dense["converged"] and red["converged"] and dense["iters"] == red["iters"]
    t = red["t"]
    assert np.max(np.abs(red["y"] - exact(t))) <= tol * np.max(np.abs(exact(t)))
    assert np.max(np.abs(dense["y"] - red["y"])) <= 1e-12 * np.max(np.abs(red["y"]))
    assert abs(red["y"][0] - q[0]) <= 1e-9 and abs(red["y"][-1] - q[1]) <= 1e-9


P15 = os.path.join(os.path.dirname(__file__), "golden", "paper_p15_B7.txt")


def p15_problem():
    """Appendix A.6's Problem 15 with its printed hyper-parameters, and the row of
    printed errors."""
    row = [line.split() for line in open(P15) if line.strip() and not line.startswith("#")][0]
    q, n, m, s2, gam = float(row[1]), int(row[2]), int(row[3]), float(row[4]), float(row[5])
    prob = dict(p=2, n=n, m=m, t0=-1.0, t1=1.0, sigma=s2 ** 0.5, gamma=gam, v=[q, q], kind="nl",
                P=[0.0, -1.0, 0.0, 0.0], delta=0.0, beta=2.0, g=0.0, omega=0.0, bc="bvp")
    return prob, tuple(float(x) for x in row[6:9])


def test_problem_15_printed_accuracy():
    """Newton on Problem 15 (f nonlinear in y') meets the printed NLS-SVM errors:
    ours within [1/10, 2] x each printed figure (ours is ~4x more accurate)."""
    from oracle import newton
    prob, printed = p15_problem()
    sol = newton.solve(prob)
    assert sol["converged"]
    e = np.abs(sol["y"] - 0.5 / np.cosh(sol["t"]))
    for ours, paper in zip((e.mean(), np.sqrt((e ** 2).mean()), e.max()), printed):
        assert paper / 10 <= ours <= 2 * paper, (ours, paper)


# ---- higher order (p = 3, 4; tabulated coefficients) -------------------------
P16 = os.path.join(os.path.dirname(__file__), "golden", "paper_p16_B7.txt")


def p16_problem():
    """Problem 16: y'''' = 120 t on [-1, 1] with y, y' at both ends, as printed."""
    row = [line.split() for line in open(P16) if line.strip() and not line.startswith("#")][0]
    n, m, s2, gam = int(row[1]), int(row[2]), float(row[3]), float(row[4])
    t = np.linspace(-1.0, 1.0, n)
    prob = dict(p=4, n=n, m=m, t0=-1.0, t1=1.0, sigma=s2 ** 0.5, gamma=gam, v=[1.0, 5.0, 3.0, 5.0],
                kind="table", f=[np.zeros(n)] * 4, r=120.0 * t, bc="bvp")
    return prob, t ** 5 + 2, tuple(float(x) for x in row[5:8])


def test_problem_16_printed_accuracy():
    """Fourth order, two conditions at each end.  As for Problems 11-13 the paper
    leaves the treatment of the numerically singular landmark kernel open; keeping
    eigenpairs down to 1e-16 lambda_max (15 of 20) gives errors within [1/10, 2] x
    the printed ones (ours ~5x smaller)."""
    prob, exact, printed = p16_problem()
    a = core.solve_linear(prob, tau=1e-16)
    b = core.solve_linear_nullspace(prob, tau=1e-16)
    e = np.abs(a["y"] - exact)
    for ours, paper in zip((e.mean(), np.sqrt((e ** 2).mean()), e.max()), printed):
        assert paper / 10 <= ours <= 2 * paper, (ours, paper)
    assert np.max(np.abs(a["y"] - b["y"])) <= 1e-10 * np.max(np.abs(a["y"]))
    assert np.max(np.abs(core.constraints(prob, a, a["omega"], a["b"]))) <= 1e-10


@pytest.mark.parametrize("p,T,sigma,m,n,tol", [(3, 3.0, 1.0, 20, 300, 5e-5), (4, 2.0, 1.0, 16, 200, 1e-3)])
def test_higher_order_ivp_closed_form(p, T, sigma, m, n, tol):
    """y''' + y' = 0 and y'''' = y with the initial values of cos t: the fit follows
    cos t and meets all p initial conditions."""
    t = np.linspace(0.0, T, n)
    z = np.zeros(n)
    f = [z, -np.ones(n), z] if p == 3 else [z, z, z, np.ones(n)]
    v = [1.0, 0.0, -1.0, 0.0][:p]
    prob = dict(p=p, n=n, m=m, t0=0.0, t1=T, sigma=sigma, gamma=1e10, v=v, kind="table", f=f, r=z)
    a = core.solve_linear(prob)
    assert np.max(np.abs(a["y"] - np.cos(t))) <= tol
    assert np.max(np.abs(core.constraints(prob, a, a["omega"], a["b"]))) <= 1e-9
    b = core.solve_linear_nullspace(prob)
    assert np.max(np.abs(a["y"] - b["y"])) <= 1e-9
