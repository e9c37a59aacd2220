"""Oracle: RBF kernel, Nystrom features and the linear primal system (Lemma 1).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

A problem is a plain dict (built by ``nys_inputs``):

    p        ODE order (1 or 2; 3 or 4 with tabulated coefficients)
    n, m     collocation points t_1..t_n (uniform on [t0, t1]) and landmarks
    t0, t1   interval
    sigma    RBF width: K(u, v) = exp(-(u - v)^2 / sigma^2)   (Section 3, RBF)
    gamma    regularisation constant
    v        initial values v_k = y^(k-1)(t_1), k = 1..p; for bc = 'bvp' the boundary
             values: y^(k)(t_1) for k < p/2, then y^(k)(t_n) for k < p/2
    bc       'ivp' (default): conditions y^(k-1)(t_1) = v_k, collocation rows 2..n
             'bvp' (p = 2 or 4): y(t_1) = q_1, y(t_n) = q_n (Appendix A.4, BVP
             case), and for p = 4 also y'(t_1), y'(t_n) (the form of Problem 16,
             Appendix B.1); collocation rows 2..n-1
    kind     'lin'   : y^(p) + sum_k a_k y^(p-k) = c sin(omega t + phi0)
             'table' : y^(p) - sum_k f_k(t) y^(p-k) = r(t), f and r given on the grid
             'nl'    : y^(p) = P(y) - delta y^(p-1) [p = 2] + g cos(omega t),
                       P(y) = c0 + c1 y + c2 y^2 + c3 y^3   (Newton, see newton.py)
    landmarks (optional) increasing indices into the grid

Readings of the paper taken here:
 * eq32 writes sqrt(m)/sqrt(eig) and a sum over a garbled index; the feature map
   used is phi(t) = Lambda^{-1/2} U^T k(t), k_j(t) = K(t, s_j), which satisfies
   phi(s_j)^T phi(s_l) = K(s_j, s_l) exactly.  The sqrt(m) variant equals the
   substitution gamma -> m * gamma (option ``scale_sqrt_m``).
 * Derivatives of the features are taken with respect to the evaluation point t
   (the first kernel argument u of the derivative formulas after Eq. 9).
 * Collocation rows are i = 2..n (the Psi matrices of Lemma 1 start at t_2);
   t_1 enters only through the initial conditions.  For the boundary value case
   of Appendix A.4 the rows are i = 2..n-1 (its Psi matrices run over
   t_2..t_{n-1}; the printed r vector ending at r(t_n) is read as ending at
   r(t_{n-1}), the same rows), and t_1, t_n enter through the two conditions.
 * Eigenpairs with eigenvalue <= tau * max eigenvalue are dropped (tau = 1e-12);
   the paper divides by sqrt(eigenvalue) and says only that they are >= 0.
 * Landmarks "evenly spaced" among the grid points (Section 4.1): index
   j -> round(j (n-1)/(m-1)), halves rounded up, both end points included.
 * The KKT matrix of Lemma 1 mixes rows of scale gamma*n with constraint rows of
   scale 1; it is solved after multiplying the constraint rows by s = max|H| and
   substituting lambda = s * lambda' (an exact transformation).
"""
import numpy as np

TAU_DEFAULT = 1e-12


# --------------------------------------------------------------------------
# grid, landmarks, kernel (Section 3; Section 4.1 sampling)
# --------------------------------------------------------------------------
def grid(prob):
    """Uniform collocation grid t_1..t_n on [t0, t1] (Section 2, problem domain)."""
    n = prob["n"]
    t0, t1 = prob["t0"], prob["t1"]
    return t0 + (t1 - t0) * np.arange(n, dtype=np.float64) / (n - 1)


def landmark_indices(prob):
    """Equidistant landmark rule (Section 4.1, 'evenly spaced'; reading above)."""
    if prob.get("landmarks") is not None:
        return np.asarray(prob["landmarks"], dtype=np.int64)
    n, m = prob["n"], prob["m"]
    idx = [(j * (n - 1) + (m - 1) // 2) // (m - 1) for j in range(m)]
    return np.asarray(idx, dtype=np.int64)


def rbf(u, v, sigma):
    """K(u, v) = exp(-(u - v)^2 / sigma^2)  (Section 3)."""
    return np.exp(-((u - v) ** 2) / sigma ** 2)


def rbf_du(u, v, sigma, ell):
    """[nabla_ell^0 K](u, v) = d^ell K / du^ell for ell = 0..4.

    Section 3: nabla_1^0 K = -2(u - v)/sigma^2 K and
    nabla_2^0 K = [4(u - v)^2/sigma^4 - 2/sigma^2] K; the third and fourth
    derivatives (higher-order ODEs, Problem 16) continue the same pattern, the
    physicists' Hermite polynomials: d^ell/du^ell K = (-1/sigma)^ell H_ell(x) K,
    x = (u - v)/sigma.
    """
    k = rbf(u, v, sigma)
    d = u - v
    s2 = sigma ** 2
    if ell == 0:
        return k
    if ell == 1:
        return -2.0 * d / s2 * k
    if ell == 2:
        return (4.0 * d ** 2 / s2 ** 2 - 2.0 / s2) * k
    if ell == 3:
        return (-8.0 * d ** 3 / s2 ** 3 + 12.0 * d / s2 ** 2) * k
    if ell == 4:
        return (16.0 * d ** 4 / s2 ** 4 - 48.0 * d ** 2 / s2 ** 3 + 12.0 / s2 ** 2) * k
    raise ValueError("derivative order > 4 is not part of the hot path")


# --------------------------------------------------------------------------
# Nystrom factor and features (Appendix A.3, eq32)
# --------------------------------------------------------------------------
def nystrom_factor(s, sigma, tau=TAU_DEFAULT):
    """Eigen-decompose the landmark kernel Omega_(m,m) (Appendix A.3).

    Returns (W, lam, U) with lam descending, eigenpairs below tau*lam_max
    dropped, and W = diag(lam)^{-1/2} U^T  (m_eff x m), so that the explicit
    feature map of eq32 is phi(t) = W k(t).
    """
    Om = rbf(s[:, None], s[None, :], sigma)
    lam, U = np.linalg.eigh(Om)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    keep = lam > tau * lam[0]
    lam, U = lam[keep], U[:, keep]
    W = (U / np.sqrt(lam)).T
    return W, lam, U


def kernel_rows(t, s, sigma, ell):
    """Matrix [nabla_ell^0 K](t_i, s_j): rows = evaluation points, cols = landmarks."""
    return rbf_du(t[:, None], s[None, :], sigma, ell)


def features(t, s, sigma, W, ell):
    """Psi^(ell) = [phi^(ell)(t_i)]_i  with phi^(ell)(t) = W k^(ell)(t)  (eq32)."""
    return kernel_rows(t, s, sigma, ell) @ W.T


# --------------------------------------------------------------------------
# ODE coefficient functions (Section 3.1: y^(p) - sum f_k y^(p-k) = r)
# --------------------------------------------------------------------------
def linear_coefficients(prob, t):
    """Return (f, r): f[k-1] = f_k(t) for k = 1..p and r(t), on the points t."""
    p = prob["p"]
    kind = prob["kind"]
    if kind == "lin":
        a = prob["a"]
        f = [np.full_like(t, -a[k]) for k in range(p)]
        r = prob["c"] * np.sin(prob["omega"] * t + prob.get("phi0", 0.0))
        return f, r
    if kind == "table":
        tt = grid(prob)
        f_tab = np.asarray(prob["f"], dtype=np.float64)
        r_tab = np.asarray(prob["r"], dtype=np.float64)
        # the table holds values on the grid; t must be grid points
        pos = np.searchsorted(tt, t)
        pos = np.clip(pos, 0, len(tt) - 1)
        if not np.allclose(tt[pos], t, rtol=0, atol=1e-12 * max(1.0, abs(tt[-1]))):
            raise ValueError("tabulated coefficients are defined on grid points only")
        return [f_tab[k][pos] for k in range(p)], r_tab[pos]
    raise ValueError("kind %r is not a linear ODE" % kind)


# --------------------------------------------------------------------------
# Collocation rows and condition rows (Section 2; Lemma 1; Appendix A.4)
# --------------------------------------------------------------------------
def is_bvp(prob):
    bc = prob.get("bc", "ivp")
    if bc not in ("ivp", "bvp"):
        raise ValueError("bc must be 'ivp' or 'bvp'")
    if bc == "bvp" and prob["p"] not in (2, 4):
        raise ValueError("boundary values: p = 2 (Appendix A.4) or p = 4 (Problem 16)")
    return bc == "bvp"


def collocation_points(prob, t):
    """Points of the collocation constraints: t_2..t_n (IVP), t_2..t_{n-1} (BVP)."""
    return t[1:-1] if is_bvp(prob) else t[1:]


def condition_rows(prob, st):
    """Rows c_k of the conditions C x = v on x = (omega, b), and v.

    IVP (Lemma 1): c_k = [phi^(k-1)(t_1), [k == 1]], v_k = y^(k-1)(t_1).
    BVP (Appendix A.4): c_1 = [phi(t_1), 1], c_2 = [phi(t_n), 1], v = (q_1, q_n);
    for p = 4 (Problem 16) the rows [phi^(k)(t_1), [k == 0]], k = 0, 1, then
    [phi^(k)(t_n), [k == 0]], k = 0, 1.
    """
    p = prob["p"]
    t, s, W = st["t"], st["s"], st["W"]
    sigma = prob["sigma"]
    me = W.shape[0]
    C = np.zeros((p, me + 1))
    if is_bvp(prob):
        h = p // 2
        for k in range(h):
            C[k, :me] = features(t[:1], s, sigma, W, k)[0]
            C[h + k, :me] = features(t[-1:], s, sigma, W, k)[0]
        C[0, me] = C[h, me] = 1.0
    else:
        for k in range(p):
            C[k, :me] = features(t[:1], s, sigma, W, k)[0]
        C[0, me] = 1.0
    return C, np.asarray(prob["v"][:p], dtype=np.float64)


# --------------------------------------------------------------------------
# Lemma 1: the primal linear system
# --------------------------------------------------------------------------
def setup(prob, tau=TAU_DEFAULT):
    """Grid, landmarks and Nystrom factor for one problem (Appendix A.3)."""
    t = grid(prob)
    idx = landmark_indices(prob)
    s = t[idx]
    W, lam, U = nystrom_factor(s, prob["sigma"], tau)
    return dict(t=t, idx=idx, s=s, W=W, lam=lam, U=U)


def lemma1_system(prob, st, gamma=None):
    """Build the (m_eff + 1 + p) square system of Lemma 1 exactly as printed.

    Psi^(l) are the feature matrices on the collocation points (t_2..t_n; for
    the BVP of Appendix A.4 t_2..t_{n-1}, whose system has the condition
    columns phi(t_1)^T, phi(t_n)^T and ones in the b row), the operator matrix is
    M = Psi^(p) - f_1 Psi^(p-1) - ... - f_p Psi (rows scaled by f_k(t_i)),
    A = gamma M^T, V = gamma (-f_p)^T, and

        [ E + A M     -A f_p    phi(t_1)^T ... phi^(p-1)(t_1)^T ] [omega ]   [A r]
        [ V M         -V f_p    1          ... 0                ] [b     ] = [V r]
        [ phi(t_1)     1        0          ... 0                ] [lam_1 ]   [v_1]
        [ phi^(k-1)(t_1) 0      0          ... 0                ] [lam_k ]   [v_k]
    """
    p = prob["p"]
    gamma = prob["gamma"] if gamma is None else gamma
    t, s, W = st["t"], st["s"], st["W"]
    sigma = prob["sigma"]
    ti = collocation_points(prob, t)
    Psi = [features(ti, s, sigma, W, ell) for ell in range(p + 1)]
    f, r = linear_coefficients(prob, ti)
    M = Psi[p].copy()
    for k in range(1, p + 1):
        M -= f[k - 1][:, None] * Psi[p - k]
    fp = f[p - 1]
    A = gamma * M.T
    V = gamma * (-fp)[None, :]
    me = W.shape[0]
    N = me + 1 + p
    K = np.zeros((N, N))
    rhs = np.zeros(N)
    K[:me, :me] = np.eye(me) + A @ M
    K[:me, me] = -(A @ fp)
    K[me, :me] = (V @ M)[0]
    K[me, me] = -(V @ fp)[0]
    C, v = condition_rows(prob, st)
    K[:me + 1, me + 1:] = C.T
    K[me + 1:, :me + 1] = C
    rhs[:me] = A @ r
    rhs[me] = (V @ r)[0]
    rhs[me + 1:] = v
    return K, rhs


def solve_kkt_scaled(K, rhs, nx):
    """Solve a KKT system [H C^T; C 0] after scaling constraint rows/cols by max|H|.

    Multiplying the constraint equations by s and writing lambda = s*lambda'
    keeps the solution exact; plain partial-pivot LU (numpy.linalg.solve)
    then sees rows of comparable size.
    """
    sc = np.abs(K[:nx, :nx]).max()
    Ks = K.copy()
    Ks[nx:, :nx] *= sc          # constraint rows times s
    Ks[:nx, nx:] *= sc          # lambda = s * lambda'
    Ks[nx:, nx:] *= sc * sc
    rs = rhs.copy()
    rs[nx:] *= sc
    sol = np.linalg.solve(Ks, rs)
    return sol[:nx], sol[nx:] * sc


def solve_linear(prob, tau=TAU_DEFAULT, st=None):
    """Solve Lemma 1 by dense LU of the printed system (primary route).

    Returns a dict with omega, b, lam (Lemma 1's sign convention), the setup
    quantities and the fitted values on the grid.
    """
    st = setup(prob, tau) if st is None else st
    gamma = prob["gamma"] * (prob["m"] if prob.get("scale_sqrt_m") else 1.0)
    K, rhs = lemma1_system(prob, st, gamma)
    me = st["W"].shape[0]
    x, lam = solve_kkt_scaled(K, rhs, me + 1)
    sol = dict(st, omega=x[:me], b=x[me], lam=lam, m_eff=me)
    sol["y"] = evaluate(prob, sol, st["t"], 0)
    return sol


def solve_linear_nullspace(prob, tau=TAU_DEFAULT, st=None):
    """Second, structurally different route to the Lemma 1 solution.

    Minimises 1/2|omega|^2 + gamma/2 sum_i e_i^2 subject to C x = v by the
    null-space method: Householder QR of C^T, the constraint part of x from R,
    the free part from a Cholesky solve of the projected Hessian.  Used only
    to cross-check ``solve_linear``.
    """
    st = setup(prob, tau) if st is None else st
    p = prob["p"]
    gamma = prob["gamma"] * (prob["m"] if prob.get("scale_sqrt_m") else 1.0)
    t, s, W = st["t"], st["s"], st["W"]
    sigma = prob["sigma"]
    ti = collocation_points(prob, t)
    f, r = linear_coefficients(prob, ti)
    # row vectors a~_i = [phi^(p) - sum f_k phi^(p-k); -f_p]
    Phi = [features(ti, s, sigma, W, ell) for ell in range(p + 1)]
    Arow = Phi[p].copy()
    for k in range(1, p + 1):
        Arow -= f[k - 1][:, None] * Phi[p - k]
    At = np.concatenate([Arow, -f[p - 1][:, None]], axis=1)
    me = W.shape[0]
    H = gamma * At.T @ At
    H[:me, :me] += np.eye(me)
    g = gamma * At.T @ r
    C, v = condition_rows(prob, st)
    Q, R = np.linalg.qr(C.T, mode="complete")
    Y, Z = Q[:, :p], Q[:, p:]
    xp = Y @ np.linalg.solve(R[:p, :p].T, v)
    L = np.linalg.cholesky(Z.T @ H @ Z)
    u = np.linalg.solve(L.T, np.linalg.solve(L, Z.T @ (g - H @ xp)))
    x = xp + Z @ u
    lam = np.linalg.solve(R[:p, :p], Y.T @ (g - H @ x))
    sol = dict(st, omega=x[:me], b=x[me], lam=lam, m_eff=me)
    sol["y"] = evaluate(prob, sol, st["t"], 0)
    return sol


def evaluate(prob, sol, tq, deriv=0):
    """Model y^(deriv)(t) = omega^T phi^(deriv)(t) + b [deriv == 0]  (Section 3)."""
    val = features(np.asarray(tq, dtype=np.float64), sol["s"], prob["sigma"],
                   sol["W"], deriv) @ sol["omega"]
    if deriv == 0:
        val = val + sol["b"]
    return val


def objective(prob, sol_like, omega, b):
    """Primal objective of Eq. 3.1.9: 1/2 |omega|^2 + gamma/2 sum_i e_i^2 over the
    collocation rows (i >= 2; i <= n-1 for the BVP).

    e_i is the residual of the collocation constraint of Section 3.1 written out
    from its definition (omega^T phi^(p) - omega^T sum f_k phi^(p-k) - f_p b - r).
    """
    p = prob["p"]
    t, s, W = sol_like["t"], sol_like["s"], sol_like["W"]
    ti = collocation_points(prob, t)
    f, r = linear_coefficients(prob, ti)
    sigma = prob["sigma"]
    lhs = features(ti, s, sigma, W, p) @ omega
    rhs_ = np.zeros_like(ti)
    for k in range(1, p + 1):
        rhs_ += f[k - 1] * (features(ti, s, sigma, W, p - k) @ omega)
    e = lhs - rhs_ - f[p - 1] * b - r
    gamma = prob["gamma"]
    return 0.5 * omega @ omega + 0.5 * gamma * np.sum(e * e)


def constraints(prob, sol_like, omega, b):
    """Condition residuals: y^(k-1)(t_1) - v_k (Section 3.1), or for the BVP
    y(t_1) - q_1 and y(t_n) - q_n (Appendix A.4)."""
    C, v = condition_rows(prob, sol_like)
    return C @ np.concatenate([omega, [b]]) - v
