"""Oracle: nonlinear ODEs by Lemma 2 (Section 3.2) and Newton's method (Eq. 3.2.1).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Problem family ('nl' in ``core``):  y^(p) = f(t, y, u), u = y^(p-1), with
    f = P(y) - delta * u + beta * u^2 / y [p = 2 only for delta, beta] + g cos(omega t),
    P(y) = c0 + c1 y + c2 y^2 + c3 y^3.
This covers y' = 1 - y^2 (tanh), the logistic equation, the Duffing equation and
the paper's Problem 15, y'' = -y + 2 (y')^2 / y (Appendix A.6).

Eq. 2.2 / Appendix A.5: unknowns (omega, b, lambda_1..lambda_p, y_2..y_n),
    L = 1/2 |omega|^2 + gamma/2 sum e_i^2 + gamma/2 sum xi_i^2 + sum_k lambda_k h_k
    e_i  = omega^T phi^(p)(t_i) - f(t_i, y_i, omega^T phi^(p-1)(t_i))
    xi_i = y_i - omega^T phi(t_i) - b
    h_1  = omega^T phi(t_1) + b - v_1,  h_2 = omega^T phi'(t_1) - v_2.
The system F = grad L = 0 (Y_1..Y_{p+3} of Lemma 2) is solved by Newton's method.
Boundary values (bc = 'bvp', p = 2; the conditions of Appendix A.4 in the
Lagrangian of its Problem 15 example): rows i = 2..n-1 and
    h_1 = omega^T phi(t_1) + b - q_1,  h_2 = omega^T phi(t_n) + b - q_n.

Readings of the paper taken here:
 * Only y_i is an auxiliary unknown; the derivative y^(p-1) inside f is
   omega^T phi^(p-1)(t_i) (as in the worked Problem 15 of Appendix A.6), so
   d e_i / d omega = phi^(p)(t_i) - f_u phi^(p-1)(t_i) changes with the iterate
   when f is nonlinear in u, and the Hessian gains - e_i f_uu phi' phi'^T and
   - e_i f_yu phi' (dropped, like - e_i f_yy, by the Gauss-Newton fallback).
 * Start: omega = 0, b = v_1, lambda = 0, y_i = v_1.  Undamped steps.
 * Full Newton; an iteration falls back to the Gauss-Newton Hessian (the
   e_i * P''(y_i) term dropped) when some diagonal entry
   d_i = gamma (P'(y_i)^2 - e_i P''(y_i) + 1) <= 1e-12 * gamma, or when the
   y-eliminated Hessian is not positive definite on the null space of the
   constraints.
 * Stop when |dx|_2 <= tol (1 + |x|_2) for x = (omega, b) and
   |F|_2 <= tol * max(1, |F(x_0)|_2); the iteration count is the number of
   Newton steps taken.
"""
import numpy as np

from . import core


def poly(prob, y):
    """P(y), P'(y), P''(y) of the polynomial part of f."""
    c0, c1, c2, c3 = prob["P"]
    P = c0 + c1 * y + c2 * y ** 2 + c3 * y ** 3
    dP = c1 + 2 * c2 * y + 3 * c3 * y ** 2
    d2P = 2 * c2 + 6 * c3 * y
    return P, dP, d2P


def rhs_f(prob, t, y, u):
    """f(t, y, u) and its partial derivatives f_y, f_u, f_yy, f_yu, f_uu."""
    P, dP, d2P = poly(prob, y)
    delta, beta = prob.get("delta", 0.0), prob.get("beta", 0.0)
    f = P - delta * u + forcing(prob, t)
    f_y, f_u, f_yy = dP, -delta + 0 * u, d2P
    f_yu = np.zeros_like(y)
    f_uu = np.zeros_like(y)
    if beta != 0.0:      # beta u^2 / y
        f = f + beta * u * u / y
        f_y = f_y - beta * u * u / y ** 2
        f_u = f_u + 2 * beta * u / y
        f_yy = f_yy + 2 * beta * u * u / y ** 3
        f_yu = -2 * beta * u / y ** 2
        f_uu = 2 * beta / y
    return f, f_y, f_u, f_yy, f_yu, f_uu


def forcing(prob, t):
    return prob.get("g", 0.0) * np.cos(prob.get("omega", 0.0) * t)


class Pieces:
    """Feature matrices of one nonlinear problem (fixed during Newton)."""

    def __init__(self, prob, tau=core.TAU_DEFAULT):
        if prob["kind"] != "nl":
            raise ValueError("newton oracle needs kind 'nl'")
        p = prob["p"]
        if p == 1 and (prob.get("delta", 0.0) != 0.0 or prob.get("beta", 0.0) != 0.0):
            raise ValueError("delta and beta terms need p = 2")
        self.prob = prob
        self.st = core.setup(prob, tau)
        st = self.st
        t, s, W = st["t"], st["s"], st["W"]
        sg = prob["sigma"]
        self.ti = core.collocation_points(prob, t)
        self.Phi = core.features(self.ti, s, sg, W, 0)
        self.Pp = core.features(self.ti, s, sg, W, p)        # phi^(p)
        self.Pu = core.features(self.ti, s, sg, W, p - 1)    # phi^(p-1): u = omega^T phi^(p-1)
        # condition rows on (omega, b) and their values
        self.C, self.v = core.condition_rows(prob, st)
        self.me = W.shape[0]
        self.p = p
        self.n1 = len(self.ti)
        self.gamma = prob["gamma"]

    # unpack x = (omega, b, lambda, y)
    def split(self, x):
        me, p = self.me, self.p
        return x[:me], x[me], x[me + 1:me + 1 + p], x[me + 1 + p:]

    def residuals(self, x):
        """e, xi, h, and per row: q = d e / d omega, f_y, f_yy, f_yu, f_uu."""
        om, b, lam, y = self.split(x)
        u = self.Pu @ om
        f, f_y, f_u, f_yy, f_yu, f_uu = rhs_f(self.prob, self.ti, y, u)
        e = self.Pp @ om - f
        xi = y - self.Phi @ om - b
        h = self.C @ np.r_[om, b] - self.v
        Q = self.Pp - f_u[:, None] * self.Pu
        return e, xi, h, Q, f_y, f_yy, f_yu, f_uu

    def lagrangian(self, x):
        """Scalar L of Appendix A.5 evaluated from its definition."""
        om, b, lam, y = self.split(x)
        e, xi, h, *_ = self.residuals(x)
        g = self.gamma
        return 0.5 * om @ om + 0.5 * g * e @ e + 0.5 * g * xi @ xi + lam @ h

    def F(self, x):
        """F = grad L = (Y_1, Y_2, Y_3..Y_{p+2}, Y_{p+3}) of Lemma 2."""
        om, b, lam, y = self.split(x)
        e, xi, h, Q, f_y, *_ = self.residuals(x)
        g = self.gamma
        me = self.me
        Y1 = om + g * Q.T @ e - g * self.Phi.T @ xi + self.C[:, :me].T @ lam
        Y2 = -g * xi.sum() + self.C[:, me] @ lam
        Yy = -g * e * f_y + g * xi
        return np.concatenate([Y1, [Y2], h, Yy])

    def diag_yy(self, x, gauss_newton):
        e, xi, h, Q, f_y, f_yy, f_yu, f_uu = self.residuals(x)
        curv = 0.0 if gauss_newton else e * f_yy
        return self.gamma * (f_y ** 2 - curv + 1.0)

    def J(self, x, gauss_newton=False):
        """Dense (m+n+p) Jacobian of F (the matrix of Lemma 2)."""
        om, b, lam, y = self.split(x)
        e, xi, h, Q, f_y, f_yy, f_yu, f_uu = self.residuals(x)
        cu = 0.0 if gauss_newton else e * f_uu       # - e f_uu phi' phi'^T
        cyu = 0.0 if gauss_newton else e * f_yu      # - e f_yu phi'
        g = self.gamma
        me, p, n1 = self.me, self.p, self.n1
        N = me + 1 + p + n1
        Jm = np.zeros((N, N))
        Jm[:me, :me] = (np.eye(me) + g * Q.T @ Q - g * (self.Pu * (cu + 0 * e)[:, None]).T @ self.Pu
                        + g * self.Phi.T @ self.Phi)
        Jm[:me, me] = g * self.Phi.sum(axis=0)
        Jm[me, :me] = Jm[:me, me]
        Jm[me, me] = g * n1
        Jm[:me + 1, me + 1:me + 1 + p] = self.C.T
        Jm[me + 1:me + 1 + p, :me + 1] = self.C
        oy = me + 1 + p
        Jwy = -g * (f_y[None, :] * Q.T + (cyu + 0 * e)[None, :] * self.Pu.T) - g * self.Phi.T   # d Y1 / d y
        Jm[:me, oy:] = Jwy
        Jm[oy:, :me] = Jwy.T
        Jm[me, oy:] = -g
        Jm[oy:, me] = -g
        Jm[oy + np.arange(n1), oy + np.arange(n1)] = self.diag_yy(x, gauss_newton)
        return Jm

    # ---- y-eliminated (Schur) form: identical Newton steps -----------------
    def reduced(self, x, gauss_newton=False):
        """Schur complement of the diagonal y-block (exact elimination).

        Returns (S, rhs_x, d, w_rows, Fy) with S the (m+1)x(m+1) reduced
        Hessian on (omega, b); the step solves [S C^T; C 0][dx; dlam] =
        [rhs_x; -h] and then dy_i = -(Fy_i + w_i^T dx) / d_i.
        """
        om, b, lam, y = self.split(x)
        e, xi, h, Q, f_y, f_yy, f_yu, f_uu = self.residuals(x)
        cu = 0.0 * e if gauss_newton else e * f_uu
        cyu = 0.0 * e if gauss_newton else e * f_yu
        g = self.gamma
        me = self.me
        Fx = self.F(x)
        Fxb = Fx[:me + 1]
        Fy = Fx[me + 1 + self.p:]
        d = self.diag_yy(x, gauss_newton)
        Qt = np.concatenate([Q, np.zeros((self.n1, 1))], axis=1)
        St = np.concatenate([self.Phi, np.ones((self.n1, 1))], axis=1)
        Ut = np.concatenate([self.Pu, np.zeros((self.n1, 1))], axis=1)
        Wr = -g * (f_y[:, None] * Qt + cyu[:, None] * Ut + St)          # rows w_i
        S = (g * Qt.T @ Qt - g * (Ut * cu[:, None]).T @ Ut + g * St.T @ St
             - (Wr / d[:, None]).T @ Wr)
        S[:me, :me] += np.eye(me)
        rhs_x = -Fxb + Wr.T @ (Fy / d)
        return S, rhs_x, d, Wr, Fy, h

    def projected_pd(self, S):
        """Is S positive definite on the null space of the constraint rows?"""
        Q, _ = np.linalg.qr(self.C.T, mode="complete")
        Z = Q[:, self.p:]
        try:
            np.linalg.cholesky(Z.T @ S @ Z)
            return True
        except np.linalg.LinAlgError:
            return False


def x0(pc):
    """Start of Newton (reading above): omega = 0, b = v_1, lambda = 0, y_i = v_1."""
    v1 = pc.v[0]
    return np.concatenate([np.zeros(pc.me), [v1], np.zeros(pc.p), np.full(pc.n1, v1)])


def use_gauss_newton(pc, x):
    d = pc.diag_yy(x, False)
    if np.any(d <= 1e-12 * pc.gamma):
        return True
    S = pc.reduced(x, False)[0]
    return not pc.projected_pd(S)


def step_dense(pc, x, gn):
    """Newton step of Eq. 3.2.1 with the dense Jacobian (constraint rows scaled)."""
    Jm = pc.J(x, gn)
    F = pc.F(x)
    me, p = pc.me, pc.p
    # move the constraint block (rows/cols me+1..me+p) to the end and scale it
    N = len(F)
    perm = np.r_[np.arange(me + 1), np.arange(me + 1 + p, N), np.arange(me + 1, me + 1 + p)]
    Jp = Jm[np.ix_(perm, perm)]
    nx = N - p
    dxp, dlam = core.solve_kkt_scaled(Jp, -F[perm], nx)
    dx = np.zeros(N)
    dx[perm[:nx]] = dxp
    dx[me + 1:me + 1 + p] = dlam
    return dx


def step_reduced(pc, x, gn):
    """The same step through the y-eliminated system (O(n m^2) per iteration)."""
    S, rhs_x, d, Wr, Fy, h = pc.reduced(x, gn)
    me, p = pc.me, pc.p
    K = np.zeros((me + 1 + p, me + 1 + p))
    K[:me + 1, :me + 1] = S
    K[:me + 1, me + 1:] = pc.C.T
    K[me + 1:, :me + 1] = pc.C
    dxb, dlam = core.solve_kkt_scaled(K, np.r_[rhs_x, -h], me + 1)
    dy = -(Fy + Wr @ dxb) / d
    return np.concatenate([dxb, dlam, dy])


def solve(prob, tol=1e-10, max_iter=50, dense=None, tau=core.TAU_DEFAULT,
          history=False):
    """Newton's method on Lemma 2's system (Eq. 3.2.1) with the stopping rule above.

    dense=None picks the dense Jacobian for n <= 600, else the reduced form.
    Returns dict(omega, b, lam, y_aux, iters, converged, y (fit on grid), ...).
    """
    pc = Pieces(prob, tau)
    if dense is None:
        dense = prob["n"] <= 600
    x = x0(pc)
    me = pc.me
    F0n = None
    dxb_prev = None
    hist = []
    converged = False
    it = 0
    for k in range(max_iter + 1):
        F = pc.F(x)
        nF = np.linalg.norm(F)
        if k == 0:
            F0n = nF
        xb = x[:me + 1]
        if history:
            hist.append(dict(x=x.copy(), nF=nF))
        if k > 0 and (np.linalg.norm(dxb_prev) <= tol * (1 + np.linalg.norm(xb))
                      and nF <= tol * max(1.0, F0n)):
            converged = True
            it = k
            break
        if k == max_iter:
            it = k
            break
        gn = use_gauss_newton(pc, x)
        dx = step_dense(pc, x, gn) if dense else step_reduced(pc, x, gn)
        x = x + dx
        dxb_prev = dx[:me + 1]
    om, b, lam, y = pc.split(x)
    sol = dict(pc.st, omega=om, b=b, lam=lam, y_aux=y, iters=it,
               converged=converged, m_eff=me, pieces=pc)
    sol["y"] = core.evaluate(prob, sol, pc.st["t"], 0)
    if history:
        sol["history"] = hist
    return sol
