"""Seeded synthetic ODE workloads (inputs only; none of the solver's arithmetic).

Both the CUDA path and the CPU oracle consume these plain problem dicts; this
module imports neither.  Every draw comes from one numpy ``Generator(PCG64)``
seeded with ``SEED`` and a per-workload spawn key, so a workload is a pure
function of its name and size arguments.

Problem dict fields (see oracle/core.py for their meaning):
    p, n, m, t0, t1, sigma, gamma, v, kind ('lin' | 'nl' | 'table') and
    kind-specific coefficients:
      lin : a = [a_1, .., a_p], c, omega, phi0   y^(p) + sum a_k y^(p-k) = c sin(omega t + phi0)
      nl  : P = [c0, c1, c2, c3], delta, g, omega y^(p) = P(y) - delta y^(p-1) + g cos(omega t)
      table: f (p x n), r (n)                    y^(p) - sum f_k y^(p-k) = r
    bc (optional): 'ivp' (default) or 'bvp' (p = 2: v = [y(t_1), y(t_n)])

The workloads mirror the paper's scales (Appendix B.5: n up to 1e4-5e4,
m = 20..200) on synthetic coefficient draws, since the paper's sixteen textbook
problems are not a dataset.
"""
import math

import numpy as np

SEED = 20251004
GAMMA = 1e10

_KEYS = {"cfg1": 1, "cfg2": 2, "m0": 10, "cfg3": 3, "cfg4": 4, "cfg5": 5, "small": 99, "trunc": 98,
         "bvp": 11, "small_bvp": 97, "small_higher": 96,
         "big_m": 95, "band": 94}


def rng(name, sub=0):
    ss = np.random.SeedSequence(SEED, spawn_key=(_KEYS[name], sub))
    return np.random.Generator(np.random.PCG64(ss))


def cfg1():
    """y'' + y = 0 on [0, 10], y(0) = 0, y'(0) = 1 (exact sin t); n=200, m=20, sigma=1, gamma=1e8."""
    return dict(p=2, n=200, m=20, t0=0.0, t1=10.0, sigma=1.0, gamma=1e8, v=[0.0, 1.0],
                kind="lin", a=[0.0, 1.0], c=0.0, omega=1.0, phi0=0.0)


def cfg2_linear(n=10_000, m=50):
    """y'' + 0.5 y' + 2 y = cos 3t on [0, 20], y(0) = 1, y'(0) = 0; sigma=0.5, gamma=1e10."""
    return dict(p=2, n=n, m=m, t0=0.0, t1=20.0, sigma=0.5, gamma=GAMMA, v=[1.0, 0.0],
                kind="lin", a=[0.5, 2.0], c=1.0, omega=3.0, phi0=math.pi / 2)


def cfg2_tanh(n=10_000, m=50):
    """y' = 1 - y^2 on [0, 5], y(0) = 0 (exact tanh t); sigma=0.5, gamma=1e10, Newton."""
    return dict(p=1, n=n, m=m, t0=0.0, t1=5.0, sigma=0.5, gamma=GAMMA, v=[0.0],
                kind="nl", P=[1.0, 0.0, -1.0, 0.0], delta=0.0, g=0.0, omega=0.0)


def linear_family(B, n=10_000, m=50, T=20.0, sigma=0.5, name="m0", sub=0, forcing="sin"):
    """B instances of y'' + a y' + b y = c sin(omega t) (or cos), n, m, sigma fixed.

    a ~ U[0,1], b ~ U[1,4], c ~ U[-1,1], omega ~ U[0.5,5], y(0), y'(0) ~ N(0,1).
    """
    g = rng(name, sub)
    a = g.uniform(0, 1, B)
    b = g.uniform(1, 4, B)
    c = g.uniform(-1, 1, B)
    w = g.uniform(0.5, 5, B)
    y0 = g.standard_normal(B)
    y1 = g.standard_normal(B)
    phi0 = 0.0 if forcing == "sin" else math.pi / 2
    return [dict(p=2, n=n, m=m, t0=0.0, t1=T, sigma=sigma, gamma=GAMMA,
                 v=[float(y0[i]), float(y1[i])], kind="lin", a=[float(a[i]), float(b[i])],
                 c=float(c[i]), omega=float(w[i]), phi0=phi0) for i in range(B)]


def m0(B=4096, n=10_000, m=50):
    """Metric batch: B instances at n = 1e4, m = 50 on [0, 20], sigma = 0.5."""
    return linear_family(B, n=n, m=m, name="m0")


def cfg3(B=4096, n_lo=500, n_hi=20_000, ms=(20, 32, 50, 64, 100)):
    """Ragged batch: T ~ U[5,30], n log-uniform in [n_lo, n_hi], m from ms, sigma = T/m."""
    g = rng("cfg3")
    T = g.uniform(5, 30, B)
    n = np.rint(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), B))).astype(int)
    m = g.choice(np.asarray(ms), B)
    a = g.uniform(0, 1, B)
    b = g.uniform(1, 4, B)
    c = g.uniform(-1, 1, B)
    w = g.uniform(0.5, 5, B)
    y0 = g.standard_normal(B)
    y1 = g.standard_normal(B)
    out = []
    for i in range(B):
        mi = int(min(m[i], n[i]))
        out.append(dict(p=2, n=int(n[i]), m=mi, t0=0.0, t1=float(T[i]), sigma=float(T[i] / mi),
                        gamma=GAMMA, v=[float(y0[i]), float(y1[i])], kind="lin",
                        a=[float(a[i]), float(b[i])], c=float(c[i]), omega=float(w[i]), phi0=0.0))
    return out


def cfg4(B=1024, n=5000, m=50, n_obs=200, noise=0.01):
    """Parameter estimation: y'' + a y' + b y = c cos(omega t) on [0, 20], sigma = 0.5.

    Returns (problems, tau [B x n_obs], y_obs [B x n_obs]); y_obs is the closed-form
    solution at sorted tau ~ U[0, 20] plus N(0, noise^2).
    """
    probs = linear_family(B, n=n, m=m, name="cfg4", forcing="cos")
    g = rng("cfg4", 1)
    tau = np.sort(g.uniform(0.0, 20.0, (B, n_obs)), axis=1)
    yobs = np.empty((B, n_obs))
    for i, pr in enumerate(probs):
        yobs[i] = closed_form_linear2(pr, tau[i]) + noise * g.standard_normal(n_obs)
    return probs, tau, yobs


def cfg5(B=64, n_lo=2000, n_hi=10_000, m=50):
    """Batched nonlinear: even index logistic y' = r y (1 - y/K), odd index Duffing.

    Duffing: y'' + delta y' + alpha y + beta y^3 = gam cos(omega t); T ~ U[5,30],
    sigma = T/m, n ~ U{n_lo..n_hi}.
    """
    g = rng("cfg5")
    out = []
    for i in range(B):
        T = float(g.uniform(5, 30))
        n = int(g.integers(n_lo, n_hi + 1))
        if i % 2 == 0:
            r = float(g.uniform(0.5, 3))
            K = float(g.uniform(1, 10))
            y0 = float(g.uniform(0.1, 1))
            out.append(dict(p=1, n=n, m=m, t0=0.0, t1=T, sigma=T / m, gamma=GAMMA, v=[y0],
                            kind="nl", P=[0.0, r, -r / K, 0.0], delta=0.0, g=0.0, omega=0.0,
                            logistic=(r, K, y0)))
        else:
            de = float(g.uniform(0.1, 0.5))
            al = float(g.uniform(-1, 1))
            be = float(g.uniform(0.5, 2))
            ga = float(g.uniform(0.2, 1))
            om = float(g.uniform(0.8, 1.5))
            y0, y1 = (float(x) for x in g.standard_normal(2))
            out.append(dict(p=2, n=n, m=m, t0=0.0, t1=T, sigma=T / m, gamma=GAMMA, v=[y0, y1],
                            kind="nl", P=[0.0, -al, 0.0, -be], delta=de, g=ga, omega=om))
    return out


def bvp_family(B, n=10_000, m=50, T=2.0, sigma=0.05, name="bvp", sub=0):
    """B boundary value problems y'' + a y' + b y = c sin(omega t), y(0) = q_1,
    y(T) = q_n (Appendix A.4 form), n, m, sigma fixed.

    a ~ U[0,1], b ~ U[-4,-1] (real characteristic roots of opposite sign: every
    instance is uniquely solvable), c ~ U[-1,1], omega ~ U[0.5,5], q ~ N(0,1).
    The metric batch rescaled to [0, 2]: the same sigma / landmark spacing and the
    same kernel band in rows.
    """
    g = rng(name, sub)
    a = g.uniform(0, 1, B)
    b = g.uniform(-4, -1, B)
    c = g.uniform(-1, 1, B)
    w = g.uniform(0.5, 5, B)
    q = g.standard_normal((B, 2))
    return [dict(p=2, n=n, m=m, t0=0.0, t1=T, sigma=sigma, gamma=GAMMA, bc="bvp",
                 v=[float(q[i, 0]), float(q[i, 1])], kind="lin", a=[float(a[i]), float(b[i])],
                 c=float(c[i]), omega=float(w[i]), phi0=0.0) for i in range(B)]


def small_bvp(B=8, sub=0, n_choices=(3, 5, 37, 64, 129, 300), m_choices=(2, 3, 5, 8, 13, 20)):
    """Small ragged boundary value problems (down to n = 3: one collocation row)."""
    g = rng("small_bvp", sub)
    out = []
    for i in range(B):
        n = int(g.choice(np.asarray(n_choices)))
        m = int(min(g.choice(np.asarray(m_choices)), n))
        T = float(g.uniform(0.5, 3))
        t0 = float(g.uniform(-1, 1))
        out.append(dict(p=2, n=n, m=m, t0=t0, t1=t0 + T, sigma=T / m * 1.5,
                        gamma=float(10 ** g.uniform(4, 10)), bc="bvp",
                        v=[float(x) for x in g.standard_normal(2)], kind="lin",
                        a=[float(g.uniform(0, 1)), float(g.uniform(-4, -1))],
                        c=float(g.uniform(-1, 1)), omega=float(g.uniform(0.5, 5)),
                        phi0=float(g.uniform(0, 3))))
    return out


def small_higher(B=8, sub=0, n_choices=(9, 37, 64, 129, 300), m_choices=(4, 7, 13, 20)):
    """Small ragged third- and fourth-order instances with tabulated coefficients
    f_k(t) = a_k + b_k sin(nu_k t) and forcing r(t) = c cos(omega t + phi0); the
    fourth-order ones take initial or boundary values (y, y' at both ends)."""
    g = rng("small_higher", sub)
    out = []
    for i in range(B):
        p = int(g.choice(np.asarray((3, 4))))
        n = int(g.choice(np.asarray(n_choices)))
        m = int(min(g.choice(np.asarray(m_choices)), n))
        T = float(g.uniform(0.5, 3))
        t0 = float(g.uniform(-1, 1))
        t = np.linspace(t0, t0 + T, n)
        f = [g.uniform(-1, 1) + g.uniform(-0.5, 0.5) * np.sin(g.uniform(0.5, 3) * t)
             for _ in range(p)]
        r = g.uniform(-1, 1) * np.cos(g.uniform(0.5, 4) * t + g.uniform(0, 3))
        out.append(dict(p=p, n=n, m=m, t0=t0, t1=t0 + T, sigma=float(T / m * g.uniform(1.5, 3)),
                        gamma=float(10 ** g.uniform(4, 10)),
                        bc="bvp" if (p == 4 and g.uniform() < 0.5) else "ivp",
                        v=[float(x) for x in g.standard_normal(p)], kind="table", f=f, r=r))
    return out


def big_m(B=6, sub=0, n_choices=(300, 701, 1500, 3000), m_choices=(113, 128, 150, 200, 224)):
    """Ragged instances with more landmarks than the shared-memory kernels hold
    (m > 112): orders 1, 2 and 4, constant or tabulated coefficients, initial or
    boundary values, kernel widths from well- to ill-conditioned landmark kernels."""
    g = rng("big_m", sub)
    out = []
    for i in range(B):
        n = int(g.choice(np.asarray(n_choices)))
        m = int(min(g.choice(np.asarray(m_choices)), n))
        p = int(g.choice(np.asarray((1, 2, 2, 4))))
        T = float(g.uniform(2, 20))
        t0 = float(g.uniform(-1, 1))
        sigma = float(T / m * g.uniform(1.0, 4.0))
        bc = "bvp" if (p in (2, 4) and g.uniform() < 0.3) else "ivp"
        q = dict(p=p, n=n, m=m, t0=t0, t1=t0 + T, sigma=sigma, gamma=float(10 ** g.uniform(5, 9)),
                 bc=bc, v=[float(x) for x in g.standard_normal(p)])
        if p == 4 or g.uniform() < 0.3:
            t = np.linspace(t0, t0 + T, n)
            q.update(kind="table",
                     f=[g.uniform(-1, 1) + g.uniform(-0.5, 0.5) * np.sin(g.uniform(0.2, 1) * t)
                        for _ in range(p)],
                     r=g.uniform(-1, 1) * np.cos(g.uniform(0.2, 2) * t + g.uniform(0, 3)))
        else:
            q.update(kind="lin", a=[float(g.uniform(0, 1)), float(g.uniform(1, 4))][:p],
                     c=float(g.uniform(-1, 1)), omega=float(g.uniform(0.2, 2)),
                     phi0=float(g.uniform(0, 3)))
        out.append(q)
    return out


def long_time(name):
    """Long-time integration workloads at the sizes of the paper's Table 12 (t up to
    100, n = 2e4 - 5e4, m = 100 - 200, gamma = 1e7), on Problems 3, 7, 8 and 9 of
    Appendix B.1, written as constant-coefficient instances:
      P3: y' + 1000 y = 1000 sin t + cos t, y(0) = 0, sigma^2 = 10, m = 200;
      P7: y'' + 0.3 y' + y = 1, y(0) = y'(0) = 0, sigma^2 = 1, m = 100;
      P8: y'' + 36 y = 0, y(0) = -1/2, y'(0) = 1, t in [0, 50], n = 2e4, m = 200;
      P9: y'' + 4 y' + 4 y = 0, y(0) = y'(0) = 1, sigma^2 = 1, m = 200.
    Returns the problem dict and its closed-form solution."""
    if name == "P3":
        return (dict(p=1, n=50000, m=200, t0=0.0, t1=100.0, sigma=10 ** 0.5, gamma=1e7, v=[0.0],
                     kind="lin", a=[1000.0], c=float(np.hypot(1000.0, 1.0)), omega=1.0,
                     phi0=float(np.arctan2(1.0, 1000.0))), lambda t: np.sin(t))
    if name == "P7":
        w = np.sqrt(1 - 0.15 ** 2)
        return (dict(p=2, n=50000, m=100, t0=0.0, t1=100.0, sigma=1.0, gamma=1e7, v=[0.0, 0.0],
                     kind="lin", a=[0.3, 1.0], c=1.0, omega=0.0, phi0=float(np.pi / 2)),
                lambda t: 1 - np.exp(-0.15 * t) * (np.cos(w * t) + 0.15 / w * np.sin(w * t)))
    if name == "P8":
        return (dict(p=2, n=20000, m=200, t0=0.0, t1=50.0, sigma=1.0, gamma=1e7, v=[-0.5, 1.0],
                     kind="lin", a=[0.0, 36.0], c=0.0, omega=0.0, phi0=0.0),
                lambda t: -0.5 * np.cos(6 * t) + np.sin(6 * t) / 6)
    if name == "P9":
        return (dict(p=2, n=50000, m=200, t0=0.0, t1=100.0, sigma=1.0, gamma=1e7, v=[1.0, 1.0],
                     kind="lin", a=[4.0, 4.0], c=0.0, omega=0.0, phi0=0.0),
                lambda t: (1 + 3 * t) * np.exp(-2 * t))
    raise KeyError(name)


def small_linear(B=8, name="small", sub=0, n_choices=(37, 64, 129, 300), m_choices=(5, 8, 13, 20),
                 p_choices=(1, 2)):
    """Small ragged linear instances (several tiles plus ragged tails) for parity tests."""
    g = rng(name, sub)
    out = []
    for i in range(B):
        p = int(g.choice(np.asarray(p_choices)))
        n = int(g.choice(np.asarray(n_choices)))
        m = int(min(g.choice(np.asarray(m_choices)), n))
        T = float(g.uniform(2, 10))
        a = [float(g.uniform(0, 1)), float(g.uniform(1, 4))][:p]
        out.append(dict(p=p, n=n, m=m, t0=float(g.uniform(-1, 1)), t1=0.0, sigma=T / m * 1.5,
                        gamma=float(10 ** g.uniform(4, 10)),
                        v=[float(x) for x in g.standard_normal(p)], kind="lin", a=a,
                        c=float(g.uniform(-1, 1)), omega=float(g.uniform(0.5, 5)),
                        phi0=float(g.uniform(0, 3))))
        out[-1]["t1"] = out[-1]["t0"] + T
    return out


# ---------------------------------------------------------------------------
# closed-form solutions (the ODEs' own, used to make observations and to check
# accuracy; they are not part of the LS-SVM method)
# ---------------------------------------------------------------------------
def closed_form_linear2(prob, t):
    """Exact solution of y'' + a y' + b y = c sin(omega t + phi0) (b > a^2/4)."""
    a, b = prob["a"]
    c, w, ph = prob["c"], prob["omega"], prob.get("phi0", 0.0)
    y0, y1 = prob["v"]
    t0 = prob["t0"]
    D = (b - w * w) ** 2 + (a * w) ** 2
    A = c * (b - w * w) / D
    Bc = c * a * w / D
    # particular solution for sin(theta), theta = w t + ph: A sin - Bc cos
    yp = lambda tt: A * np.sin(w * tt + ph) - Bc * np.cos(w * tt + ph)          # noqa: E731
    ypd = lambda tt: A * w * np.cos(w * tt + ph) + Bc * w * np.sin(w * tt + ph)  # noqa: E731
    beta = math.sqrt(b - a * a / 4)
    C1 = y0 - yp(t0)
    C2 = (y1 - ypd(t0) + a / 2 * C1) / beta
    s = np.asarray(t) - t0
    return np.exp(-a * s / 2) * (C1 * np.cos(beta * s) + C2 * np.sin(beta * s)) + yp(np.asarray(t))


def closed_form_logistic(prob, t):
    r, K, y0 = prob["logistic"]
    return K / (1 + (K / y0 - 1) * np.exp(-r * (np.asarray(t) - prob["t0"])))
