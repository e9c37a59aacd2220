"""Pins of the oracle's linear path against things other than itself.

Kernel derivatives vs finite differences and Hermite polynomials, exact Nystrom
identities, the printed accuracy of the paper (table in Appendix B.7), closed-form ODE
solutions, brute-force optimality of the primal problem, invariances.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite as H

import nys_inputs as ni
from oracle import core, dual

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_B7.txt")


# ---------------------------------------------------------------- kernel ----
@pytest.mark.parametrize("sigma", [0.3, 1.0, 3.0])
def test_kernel_derivatives_match_finite_differences(sigma):
    u = np.linspace(-3 * sigma, 3 * sigma, 41) + 0.123
    v = 0.37
    h = 1e-4 * sigma
    for ell in (1, 2, 3, 4):
        fd = (core.rbf_du(u + h, v, sigma, ell - 1) - core.rbf_du(u - h, v, sigma, ell - 1)) / (2 * h)
        an = core.rbf_du(u, v, sigma, ell)
        assert np.max(np.abs(fd - an)) <= 1e-7 * np.max(np.abs(an)) * (1 / sigma + 1)


@pytest.mark.parametrize("sigma", [0.5, 2.0])
def test_kernel_derivatives_are_hermite_multiples(sigma):
    """d^q/dd^q exp(-(d/s)^2) = (-1/s)^q H_q(d/s) exp(-(d/s)^2), physicists' Hermite."""
    d = np.linspace(-4, 4, 33)
    x = d / sigma
    base = np.exp(-x * x)
    for q in range(0, 5):
        coef = np.zeros(q + 1)
        coef[q] = 1
        ref = (-1.0 / sigma) ** q * H.hermval(x, coef) * base
        np.testing.assert_allclose(core.rbf_du(d, 0.0, sigma, q), ref, atol=1e-13 * np.abs(ref).max())
        for a in range(q + 1):
            c = q - a
            got = dual.rbf_mixed(d, 0.0, sigma, a, c)
            np.testing.assert_allclose(got, (-1) ** c * ref, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------- landmarks --
@pytest.mark.parametrize("n,m", [(200, 20), (10_000, 50), (37, 5), (16, 16), (101, 2)])
def test_landmark_rule_evenly_spaced(n, m):
    idx = core.landmark_indices(dict(n=n, m=m))
    assert idx[0] == 0 and idx[-1] == n - 1 and len(idx) == m
    gaps = np.diff(idx)
    assert gaps.min() >= math.floor((n - 1) / (m - 1)) and gaps.max() <= math.ceil((n - 1) / (m - 1))
    exact = np.arange(m) * (n - 1) / (m - 1)
    assert np.all(np.abs(idx - exact) <= 0.5)


# ---------------------------------------------------------------- Nystrom ----
def test_features_reproduce_landmark_kernel():
    prob = ni.cfg2_linear(n=2000, m=50)
    st = core.setup(prob)
    Phi = core.features(st["s"], st["s"], prob["sigma"], st["W"], 0)
    Om = core.rbf(st["s"][:, None], st["s"][None, :], prob["sigma"])
    assert st["W"].shape[0] == 50
    np.testing.assert_allclose(Phi @ Phi.T, Om, atol=1e-12)


def test_m_equals_n_reproduces_full_kernel_and_its_derivative():
    """All grid points as landmarks: phi^(l)(t)^T phi(t_j) = d^l/dt^l K(t, t_j)."""
    prob = dict(n=12, m=12, t0=0.0, t1=5.5, sigma=0.8)
    t = core.grid(prob)
    st = dict(t=t, s=t, **dict(zip(("W", "lam", "U"), core.nystrom_factor(t, prob["sigma"]))))
    assert st["W"].shape[0] == 12
    tq = np.array([0.1, 1.234, 2.5, 4.9])
    Pj = core.features(t, t, prob["sigma"], st["W"], 0)
    for ell in (0, 1, 2):
        Pq = core.features(tq, t, prob["sigma"], st["W"], ell)
        ref = core.rbf_du(tq[:, None], t[None, :], prob["sigma"], ell)
        np.testing.assert_allclose(Pq @ Pj.T, ref, atol=1e-9 * np.abs(ref).max())


def test_feature_derivatives_match_finite_differences():
    prob = ni.cfg1()
    st = core.setup(prob)
    tq = np.linspace(0.05, 9.9, 57)
    h = 1e-5
    for ell in (1, 2):
        fd = (core.features(tq + h, st["s"], 1.0, st["W"], ell - 1)
              - core.features(tq - h, st["s"], 1.0, st["W"], ell - 1)) / (2 * h)
        an = core.features(tq, st["s"], 1.0, st["W"], ell)
        assert np.max(np.abs(fd - an)) <= 1e-7 * np.max(np.abs(an))


def test_small_eigenvalues_are_truncated():
    prob = dict(n=1000, m=50, t0=0.0, t1=2.0, sigma=1.0)   # Problem 8 scale: Omega singular
    st = core.setup(prob)
    assert 5 < st["W"].shape[0] < 50
    assert st["lam"].min() > 1e-12 * st["lam"].max()


# ---------------------------------------------------------------- Lemma 1 ----
def _cases():
    return [ni.cfg1(), ni.cfg2_linear(n=3000)] + ni.small_linear(4)


@pytest.mark.parametrize("k", range(6))
def test_dense_lu_and_null_space_routes_agree(k):
    prob = _cases()[k]
    a = core.solve_linear(prob)
    b = core.solve_linear_nullspace(prob)
    sc = np.abs(a["y"]).max()
    assert np.abs(a["y"] - b["y"]).max() <= 1e-10 * sc
    assert abs(a["b"] - b["b"]) <= 1e-9 * max(1.0, abs(a["b"]))
    np.testing.assert_allclose(a["lam"], b["lam"], rtol=1e-7, atol=1e-9 * np.abs(a["lam"]).max())


@pytest.mark.parametrize("k", range(6))
def test_solution_meets_initial_conditions(k):
    prob = _cases()[k]
    sol = core.solve_linear(prob)
    res = core.constraints(prob, sol, sol["omega"], sol["b"])
    assert np.all(np.abs(res) <= 1e-9 * (1 + np.abs(prob["v"]).max()))


@pytest.mark.parametrize("k", [0, 2, 3])
def test_solution_minimises_the_primal_objective(k):
    """Brute force: no feasible perturbation lowers the objective of Eq. 3.1.9."""
    prob = _cases()[k]
    if prob["gamma"] > 1e8:
        prob = dict(prob, gamma=1e6)
    sol = core.solve_linear(prob)
    me = sol["m_eff"]
    p = prob["p"]
    C = np.zeros((p, me + 1))
    for j in range(p):
        C[j, :me] = core.features(sol["t"][:1], sol["s"], prob["sigma"], sol["W"], j)[0]
    C[0, me] = 1.0
    Q, _ = np.linalg.qr(C.T, mode="complete")
    Z = Q[:, p:]
    x = np.r_[sol["omega"], sol["b"]]
    J0 = core.objective(prob, sol, sol["omega"], sol["b"])
    rng = np.random.default_rng(k)
    for _ in range(5):
        d = Z @ rng.standard_normal(Z.shape[1])
        d /= np.linalg.norm(d)
        for eps in (1e-3, 1e-2):
            xp = x + eps * d * max(1.0, np.linalg.norm(x))
            assert core.objective(prob, sol, xp[:me], xp[me]) >= J0 * (1 - 1e-12)
        # stationarity: central difference of J along d vanishes relative to the curvature
        e = 1e-4 * max(1.0, np.linalg.norm(x))
        Jp = core.objective(prob, sol, (x + e * d)[:me], (x + e * d)[me])
        Jm = core.objective(prob, sol, (x - e * d)[:me], (x - e * d)[me])
        slope = (Jp - Jm) / (2 * e)
        curv = (Jp - 2 * J0 + Jm) / e ** 2
        assert abs(slope) <= 1e-5 * max(curv * np.linalg.norm(x), 1.0)


def test_rotation_of_features_leaves_fit_unchanged():
    prob = ni.cfg2_linear(n=2000)
    st = core.setup(prob)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((st["W"].shape[0],) * 2))
    st2 = dict(st, W=Q @ st["W"])
    a = core.solve_linear(prob, st=st)
    b = core.solve_linear(prob, st=st2)
    assert np.abs(a["y"] - b["y"]).max() <= 1e-10 * np.abs(a["y"]).max()


def test_cholesky_whitening_gives_the_same_fit():
    """Any W with W^T W = Omega^-1 spans the same features up to an orthogonal map,
    so W = L^-1 (Omega = L L^T) fits exactly like Appendix A.3's Lambda^-1/2 U^T when
    nothing is truncated (the GPU setup uses it when cond(Omega) is small)."""
    for prob in (ni.cfg2_linear(n=2000), ni.cfg1(), ni.m0(1, n=3000)[0]):
        st = core.setup(prob)
        assert st["W"].shape[0] == prob["m"]
        t = core.grid(prob)
        s = t[core.landmark_indices(prob)]
        L = np.linalg.cholesky(core.rbf(s[:, None], s[None, :], prob["sigma"]))
        Wc = np.linalg.solve(L, np.eye(len(s)))
        a = core.solve_linear(prob, st=st)
        b = core.solve_linear(prob, st=dict(st, W=Wc))
        assert np.abs(a["y"] - b["y"]).max() <= 1e-10 * np.abs(a["y"]).max()
        assert abs(a["b"] - b["b"]) <= 1e-10 * max(1.0, np.abs(a["y"]).max())


def test_sqrt_m_feature_scaling_equals_gamma_times_m():
    prob = ni.cfg1()
    st = core.setup(prob)
    st_scaled = dict(st, W=math.sqrt(prob["m"]) * st["W"])
    a = core.solve_linear(prob, st=st_scaled)            # eq32 as printed (sqrt(m) factor)
    b = core.solve_linear(dict(prob, scale_sqrt_m=True))  # option used by the library
    assert np.abs(a["y"] - b["y"]).max() <= 1e-10 * np.abs(a["y"]).max()


def test_primal_equals_dual_with_nystrom_kernel():
    """Lagrange dual with K~ = k^T Omega^+ k (never forms features): same fit."""
    for prob in (dict(ni.cfg1(), n=120, gamma=1e4), dict(ni.small_linear(3)[1], gamma=1e4)):
        a = core.solve_linear(prob)
        d = dual.solve_dual(prob, "nystrom")
        assert np.abs(a["y"] - d["y"]).max() <= 1e-9 * np.abs(a["y"]).max()
        assert abs(a["b"] - d["b"]) <= 1e-8 * max(1, abs(a["b"]))


def test_classical_lssvm_and_nystrom_both_solve_cfg1():
    prob = ni.cfg1()
    a = core.solve_linear(prob)
    d = dual.solve_dual(prob, "rbf")
    t = a["t"]
    assert np.abs(d["y"] - np.sin(t)).max() < 1e-4      # classical LS-SVM, n = 200
    assert np.abs(a["y"] - np.sin(t)).max() < 5e-2      # Nystrom, only m = 20 features


# ------------------------------------------------------ accuracy vs truth ----
def test_closed_form_second_order_linear():
    prob = dict(ni.cfg2_linear(), sigma=1.0)   # resolved width for this interval
    sol = core.solve_linear(prob)
    err = np.abs(sol["y"] - ni.closed_form_linear2(prob, sol["t"])).max()
    assert err < 2e-3
    for prob in ni.m0(3):
        prob = dict(prob, sigma=1.0)
        sol = core.solve_linear(prob)
        ex = ni.closed_form_linear2(prob, sol["t"])
        assert np.abs(sol["y"] - ex).max() < 3e-2 * np.abs(ex).max()


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0],) + tuple(float(x) for x in f[1:]))
    return rows


def _exact(name, t):
    if name == "P7":
        bt = math.sqrt(1 - 0.15 ** 2)
        return 1 - np.exp(-0.15 * t) * (np.cos(bt * t) + 0.15 / bt * np.sin(bt * t))
    if name == "P8":
        return -0.5 * np.cos(6 * t) + np.sin(6 * t) / 6
    if name == "P9":
        return (1 + 3 * t) * np.exp(-2 * t)
    raise KeyError(name)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_paper_table_B7_accuracy(row):
    """The paper's printed NLS-SVM errors are matched to within the freedom the paper
    leaves open (landmark positions, handling of the numerically singular landmark
    kernel): ours is at most 2x each printed figure and, for P7 and P9, at least 1/10
    of it.  For P8 (t in [0, 2], 50 landmarks with sigma = 1: only 12 eigenpairs above
    1e-12) our fit is ~80x more accurate than printed, so only the upper bound applies."""
    name, a1, a2, rc, t0, t1, y0, y0p, n, m, s2, gam, mae, rmse, linf = row
    prob = dict(p=2, n=int(n), m=int(m), t0=t0, t1=t1, sigma=math.sqrt(s2), gamma=gam,
                v=[y0, y0p], kind="lin", a=[a1, a2], c=rc, omega=0.0, phi0=math.pi / 2)
    sol = core.solve_linear(prob)
    e = np.abs(sol["y"] - _exact(name, sol["t"]))
    for ours, paper in ((e.mean(), mae), (np.sqrt((e ** 2).mean()), rmse), (e.max(), linf)):
        assert ours <= 2 * paper, (name, ours, paper)
        if name != "P8":
            assert ours >= paper / 10, (name, ours, paper)


def test_metric_configuration_equals_constrained_least_squares_collocation():
    """When no eigenpair is dropped (m_eff = m) the Nystrom features span the landmark
    kernels k(., s_j), so as gamma grows Lemma 1's primal problem tends to the
    equality-constrained least-squares collocation
        min_z |A z - r|^2  s.t.  y(t_1) = v_1, y'(t_1) = v_2,
    over y = sum_j z_j k(t, s_j) + b, A the operator y'' + a y' + b y on rows 2..n.
    Built here from the definitions alone: the uniform grid, landmark indices
    round(j (n-1) / (m-1)), kernel exp(-d^2/sigma^2) and its t-derivatives, a
    KKT solve by numpy's lstsq.  At the metric configuration (n = 1e4, m = 50,
    sigma = 0.5, gamma = 1e10) the oracle's fit matches it to <= 1e-12 (measured
    3e-13 .. 1e-12).  At this sigma, 1.2 landmark spacings, the method's fit is
    15-41 % from the ODE's exact solution.  That is the span's limit: its best
    approximation of the exact y has a y'' residual of 7.5.  It is not an oracle
    error."""
    for q in ni.m0(2):
        n, m, sig = q["n"], q["m"], q["sigma"]
        t = np.linspace(q["t0"], q["t1"], n)
        s = t[[(j * (n - 1) * 2 + (m - 1)) // (2 * (m - 1)) for j in range(m)]]
        d = t[:, None] - s[None, :]
        e = np.exp(-d ** 2 / sig ** 2)
        k1, k2 = -2 * d / sig ** 2 * e, (4 * d ** 2 / sig ** 4 - 2 / sig ** 2) * e
        a1, b1 = q["a"]
        r = q["c"] * np.sin(q["omega"] * t + q["phi0"])
        A = np.c_[k2 + a1 * k1 + b1 * e, b1 * np.ones(n)][1:]
        C = np.vstack([np.r_[e[0], 1.0], np.r_[k1[0], 0.0]])
        M = np.block([[A.T @ A, C.T], [C, np.zeros((2, 2))]])
        z = np.linalg.lstsq(M, np.r_[A.T @ r[1:], q["v"]], rcond=None)[0][:m + 1]
        y_ls = np.c_[e, np.ones(n)] @ z
        sol = core.solve_linear(q)
        assert sol["m_eff"] == m
        assert np.abs(sol["y"] - y_ls).max() <= 1e-12 * np.abs(y_ls).max()
