"""Oracle checks: dual LS-SVM formulations of the linear ODE problem.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The primal problem of Lemma 1 (Section 3.1) is a regularised least-squares fit
with equality constraints.  Its Lagrange dual (the route of the classical
LS-SVM ODE solver, Appendix A.1 and Mehrkanoon et al.) needs only kernel values
K~(u, v) = phi(u)^T phi(v) and their derivatives, never the feature vectors:

    a_i = phi^(p)(t_i) - sum_k f_k(t_i) phi^(p-k)(t_i),  i = 2..n
    omega = sum_i alpha_i a_i + sum_k beta_k phi^(k-1)(t_1)
    [ G + I/gamma   B      -f_p ] [alpha]   [r]
    [ B^T           Cc     e_1  ] [beta ] = [v]
    [ -f_p^T        e_1^T   0   ] [b    ]   [0]
with G_ij = a_i^T a_j, B_ik = a_i^T phi^(k-1)(t_1), Cc_kl = phi^(k-1)(t_1)^T phi^(l-1)(t_1).

With the Nystrom kernel K~(u, v) = k(u)^T Omega^+ k(v) (Omega^+ the truncated
pseudo-inverse of the landmark kernel, eq32) this dual has exactly the primal
solution; with the true RBF kernel it is the classical LS-SVM, which the paper
compares against (Section 5: within 0.13 % relative).  O(n^3): small n only.
"""
import numpy as np

from . import core


def rbf_mixed(u, v, sigma, a, c):
    """d^{a+c} K / du^a dv^c for the RBF kernel, a + c <= 4 (Eq. 9 operator).

    K depends on d = u - v only, so d/dv = -d/dd; the d-derivatives of
    exp(-d^2/sigma^2) are Hermite-polynomial multiples of the kernel.
    """
    d = u - v
    s2 = sigma ** 2
    k = np.exp(-d ** 2 / s2)
    q = a + c
    if q == 0:
        g = k
    elif q == 1:
        g = -2 * d / s2 * k
    elif q == 2:
        g = (4 * d ** 2 / s2 ** 2 - 2 / s2) * k
    elif q == 3:
        g = (-8 * d ** 3 / s2 ** 3 + 12 * d / s2 ** 2) * k
    elif q == 4:
        g = (16 * d ** 4 / s2 ** 4 - 48 * d ** 2 / s2 ** 3 + 12 / s2 ** 2) * k
    else:
        raise ValueError("order > 4")
    return (-1) ** c * g


def _kernel_block(kfun, prob, t_rows, t_cols, a_row, a_col):
    """sum_{a,c} w_a(row) w_c(col) d^{a+c}K(t_r, t_c) for operator weights."""
    out = np.zeros((len(t_rows), len(t_cols)))
    for a, wa in a_row:
        for c, wc in a_col:
            out += wa[:, None] * wc[None, :] * kfun(t_rows[:, None], t_cols[None, :], a, c)
    return out


def solve_dual(prob, kernel="nystrom", tau=core.TAU_DEFAULT):
    """Solve the dual system above; return fitted values on the grid and b."""
    p = prob["p"]
    st = core.setup(prob, tau)
    t, s, U, lam = st["t"], st["s"], st["U"], st["lam"]
    sigma = prob["sigma"]
    gamma = prob["gamma"]
    if kernel == "nystrom":
        Op = (U / lam) @ U.T

        # explicit: K~^(a,c)(u, v) = k^(a)(u)^T Omega^+ k^(c)(v)
        def kfun(u, v, a, c):
            uu = u[:, 0]
            vv = v[0, :]
            ka = core.kernel_rows(uu, s, sigma, a)
            kc = core.kernel_rows(vv, s, sigma, c)
            return ka @ Op @ kc.T
    elif kernel == "rbf":
        def kfun(u, v, a, c):
            return rbf_mixed(u, v, sigma, a, c)
    else:
        raise ValueError(kernel)

    ti = t[1:]
    f, r = core.linear_coefficients(prob, ti)
    # operator on the collocation rows: y^(p) - sum_k f_k y^(p-k)
    op_rows = [(p, np.ones_like(ti))] + [(p - k, -f[k - 1]) for k in range(1, p + 1)]
    t1 = t[:1]
    n1 = len(ti)
    G = _kernel_block(kfun, prob, ti, ti, op_rows, op_rows)
    B = np.zeros((n1, p))
    Cc = np.zeros((p, p))
    for k in range(p):
        B[:, k] = _kernel_block(kfun, prob, ti, t1, op_rows, [(k, np.ones(1))])[:, 0]
        for l in range(p):
            Cc[k, l] = _kernel_block(kfun, prob, t1, t1, [(k, np.ones(1))],
                                     [(l, np.ones(1))])[0, 0]
    N = n1 + p + 1
    K = np.zeros((N, N))
    K[:n1, :n1] = G + np.eye(n1) / gamma
    K[:n1, n1:n1 + p] = B
    K[n1:n1 + p, :n1] = B.T
    K[n1:n1 + p, n1:n1 + p] = Cc
    K[:n1, -1] = -f[p - 1]
    K[-1, :n1] = -f[p - 1]
    K[n1, -1] = 1.0
    K[-1, n1] = 1.0
    rhs = np.concatenate([r, np.asarray(prob["v"][:p], dtype=np.float64), [0.0]])
    sol = np.linalg.solve(K, rhs)
    alpha, beta, b = sol[:n1], sol[n1:n1 + p], sol[-1]
    # y(t) = sum_j alpha_j L_v K(t, t_j) + sum_k beta_k d^{k-1}_v K(t, t_1) + b
    y = _kernel_block(kfun, prob, t, ti, [(0, np.ones_like(t))], op_rows) @ alpha
    for k in range(p):
        y += _kernel_block(kfun, prob, t, t1, [(0, np.ones_like(t))],
                           [(k, np.ones(1))])[:, 0] * beta[k]
    y += b
    return dict(y=y, b=b, alpha=alpha, beta=beta, t=t)
