"""Problems 11-13 of the paper's benchmark list (Appendix B.1), linear second-order
boundary value problems on [0, 1], as problem dicts with tabulated coefficients,
plus their printed NLS-SVM errors (golden fixture).  Shared by the oracle pins and
the GPU parity tests."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_bvp_B7.txt")


def golden_rows():
    """(name, q1, qn, n, m, sigma2, gamma, MAE, RMSE, Linf) per problem."""
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0],) + tuple(float(x) for x in f[1:]))
    return rows


def problem(name, q1, qn, n, m, s2, gam):
    """y'' = f1 y' + f2 y + r, y(0) = q1, y(1) = qn, tabulated on the grid, and the
    analytical solution there.  The coefficients are singular at t = 0 = t_1, which
    is not a collocation point; the table holds 0 there."""
    n, m = int(n), int(m)
    t = np.linspace(0.0, 1.0, n)
    ts = np.where(t == 0, 1.0, t)
    z = t == 0
    if name == "P11":     # y'' + y'/t + cos t + sin(t)/t = 0, y = cos t
        f1, f2, r = np.where(z, 0, -1 / ts), np.zeros(n), np.where(z, 0, -np.cos(t) - np.sin(t) / ts)
        exact = np.cos(t)
    elif name == "P12":   # y'' + y = 2
        f1, f2, r = np.zeros(n), -np.ones(n), 2.0 * np.ones(n)
        exact = 2 - np.cos(t) + (math.cos(1) - 2) / math.sin(1) * np.sin(t)
    elif name == "P13":   # y'' + (1-2t)/t y' + (t-1)/t y = 0, y = e^t
        f1, f2, r = np.where(z, 0, -(1 - 2 * t) / ts), np.where(z, 0, -(t - 1) / ts), np.zeros(n)
        exact = np.exp(t)
    else:
        raise KeyError(name)
    prob = dict(p=2, n=n, m=m, t0=0.0, t1=1.0, sigma=math.sqrt(s2), gamma=gam, v=[q1, qn],
                kind="table", f=[f1, f2], r=r, bc="bvp")
    return prob, exact


def problems():
    return [problem(*row[:7]) for row in golden_rows()]
