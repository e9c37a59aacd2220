"""Oracle: gradients of a loss on the fitted solution (parameter-estimation use).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper cites parameter estimation as a use of LS-SVM ODE solvers
(Introduction, Mehrkanoon et al. 2014) but gives no gradient formula.  The
gradient here is d loss / d theta for theta = (a, b, c, omega, y0, y0', sigma) of

    y'' + a y' + b y = c sin(omega t + phi0),  y(t_1) = y0,  y'(t_1) = y0'

with the loss evaluated on the fitted model y^(tau_j) at observation times.

Route: the fitted values do not depend on the orthogonal basis of the Nystrom
features, so with all eigenpairs kept (m_eff = m) the problem of Lemma 1 equals
the kernel-coordinate problem in z = (alpha, b) with alpha = W^T omega:

    min 1/2 alpha^T Omega alpha + gamma/2 sum_i (kappa_i^T alpha + a_p b - r_i)^2
    s.t. alpha^T k(t_1) + b = y0,  alpha^T k'(t_1) = y0'
    kappa_i = k''(t_i) + a k'(t_i) + b k(t_i)      (p = 2; p = 1 analogous)

which involves kernel values only.  It is differentiated by the complex-step
method (Squire & Trapp 1998): d l/d theta = Im l(theta + i h) / h, h = 1e-30,
exact to rounding for this real-analytic map.  ``fd_gradient`` gives central
finite differences of the eigen-route oracle (core.solve_linear) instead.
"""
import numpy as np

from . import core

PARAMS = ("a", "b", "c", "omega", "y0", "y0p", "sigma")


def _unpack(prob):
    p = prob["p"]
    a = list(prob["a"]) + [0.0] * (2 - p)
    return dict(a=a[0], b=a[1], c=prob["c"], omega=prob["omega"], y0=prob["v"][0],
                y0p=prob["v"][1] if p == 2 else 0.0, sigma=prob["sigma"])


def _repack(prob, th):
    q = dict(prob)
    p = prob["p"]
    q["a"] = [th["a"], th["b"]][:p]
    q["c"] = th["c"]
    q["omega"] = th["omega"]
    q["v"] = [th["y0"], th["y0p"]][:p]
    q["sigma"] = th["sigma"]
    return q


def _k(t, s, sigma, ell):
    """Kernel derivative rows, complex-safe (same formulas as core.rbf_du)."""
    d = t[:, None] - s[None, :]
    k = np.exp(-d ** 2 / sigma ** 2)
    if ell == 0:
        return k
    if ell == 1:
        return -2.0 * d / sigma ** 2 * k
    return (4.0 * d ** 2 / sigma ** 4 - 2.0 / sigma ** 2) * k


def solve_kernel_coords(prob, th=None):
    """Solve the kernel-coordinate problem above (complex-capable). Returns z, lam, s."""
    th = _unpack(prob) if th is None else th
    p = prob["p"]
    t = core.grid(prob)
    s = t[core.landmark_indices(prob)]
    sg = th["sigma"]
    ti = t[1:]
    a_coef = [th["a"], th["b"]][:p]            # y^(p) + sum a_k y^(p-k)
    kap = _k(ti, s, sg, p).astype(complex)
    for k in range(1, p + 1):
        kap = kap + a_coef[k - 1] * _k(ti, s, sg, p - k)
    m = len(s)
    n1 = len(ti)
    kt = np.concatenate([kap, np.full((n1, 1), a_coef[p - 1], dtype=complex)], axis=1)
    r = th["c"] * np.sin(th["omega"] * ti + prob.get("phi0", 0.0))
    gamma = prob["gamma"]
    M = gamma * kt.T @ kt
    M[:m, :m] += _k(s, s, sg, 0)
    g = gamma * kt.T @ r
    E = np.zeros((p, m + 1), dtype=complex)
    E[0, :m] = _k(t[:1], s, sg, 0)[0]
    E[0, m] = 1.0
    if p == 2:
        E[1, :m] = _k(t[:1], s, sg, 1)[0]
    v = np.array([th["y0"], th["y0p"]][:p], dtype=complex)
    sc = np.abs(M.real).max()
    K = np.zeros((m + 1 + p, m + 1 + p), dtype=complex)
    K[:m + 1, :m + 1] = M
    K[:m + 1, m + 1:] = sc * E.T
    K[m + 1:, :m + 1] = sc * E
    sol = np.linalg.solve(K, np.concatenate([g, sc * v]))
    return sol[:m + 1], sol[m + 1:] * sc, s


def fitted(prob, tq, th=None):
    """y^(tau) = alpha^T k(tau) + b of the kernel-coordinate solution."""
    th = _unpack(prob) if th is None else th
    z, lam, s = solve_kernel_coords(prob, th)
    m = len(s)
    return _k(np.asarray(tq, dtype=np.float64), s, th["sigma"], 0) @ z[:m] + z[m]


def mse_loss(yhat, yobs):
    d = yhat - yobs
    return np.sum(d * d) / len(yobs)


def complex_step_gradient(prob, tq, yobs, loss=mse_loss, h=1e-30):
    """d loss(y^(tq)) / d theta for theta in PARAMS, by complex step."""
    th0 = _unpack(prob)
    out = np.zeros(len(PARAMS))
    for j, name in enumerate(PARAMS):
        th = {k: complex(v) for k, v in th0.items()}
        th[name] = th[name] + 1j * h
        out[j] = loss(fitted(prob, tq, th), yobs).imag / h
    return out


def fd_gradient(prob, tq, yobs, loss=mse_loss, rel=1e-6):
    """Central finite differences of the eigen-route oracle (core.solve_linear)."""
    th0 = _unpack(prob)
    out = np.zeros(len(PARAMS))
    for j, name in enumerate(PARAMS):
        hstep = rel * max(1.0, abs(th0[name]))
        vals = []
        for sgn in (+1, -1):
            th = dict(th0)
            th[name] = th0[name] + sgn * hstep
            q = _repack(prob, th)
            sol = core.solve_linear(q)
            vals.append(loss(core.evaluate(q, sol, tq, 0), yobs))
        out[j] = (vals[0] - vals[1]) / (2 * hstep)
    return out
