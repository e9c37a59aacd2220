"""GPU parity of the boundary value case (Appendix A.4: y(t_1) = q_1, y(t_n) = q_n,
collocation rows 2..n-1) against the FP64 oracle, through the C ABI.

Tolerances as for initial value problems: max|y_gpu - y_oracle| / max|y_oracle|
<= 1e-10 (FP64) and <= 1e-6 (mixed), or 10x the spread between the oracle's own two
exact routes where the problem itself is that sensitive (tiny degenerate cases and
the truncated landmark kernels of Problems 11-13)."""
import ctypes as C

import numpy as np
import pytest

import nys_inputs as ni
from oracle import core

from bvp_problems import problems as paper_problems

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-6}


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_04094_gb300 import api as A
    return A


def _check(api, probs, precision):
    import torch
    bt = api.Batch(probs, precision=precision)
    bt.assemble()
    x, st = bt.solve()
    grids = [core.grid(q) for q in probs]
    y, _ = bt.eval(grids)
    y1, _ = bt.eval(grids, deriv=1)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert (st == 0).all(), st
    meff = bt.m_eff()
    sols = bt.unpack()
    yc, y1c = y.cpu().numpy(), y1.cpu().numpy()
    off = 0
    for k, (q, g) in enumerate(zip(probs, grids)):
        ref = core.solve_linear(q)
        ref2 = core.solve_linear_nullspace(q)
        scale = np.abs(ref["y"]).max()
        tol = max(TOL[precision], 10 * np.abs(ref["y"] - ref2["y"]).max() / scale)
        # b alone can be ill-determined (smooth features nearly span the constants:
        # the oracle's own routes differ by 2e-4 on Problem 11 while y agrees)
        tol_b = max(10 * tol, 10 * abs(ref["b"] - ref2["b"]) / max(1.0, scale))
        assert meff[k] == ref["m_eff"]
        got = yc[off:off + len(g)]
        err = np.abs(got - ref["y"]).max() / scale
        d1 = core.evaluate(q, ref, g, 1)
        err1 = np.abs(y1c[off:off + len(g)] - d1).max() / np.abs(d1).max()
        eb = abs(sols[k]["b"] - ref["b"]) / max(1.0, scale)
        assert err <= tol, (k, q["n"], q["m"], err, tol)
        assert err1 <= 50 * tol, (k, err1)
        assert eb <= tol_b, (k, eb, tol_b)
        if q.get("bc") == "bvp":   # the boundary values themselves
            assert abs(got[0] - q["v"][0]) <= 10 * tol * max(1.0, scale)
            assert abs(got[-1] - q["v"][1]) <= 10 * tol * max(1.0, scale)
        off += len(g)
    bt.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_ragged_bvp_batch(api, precision):
    """n from 3 (one collocation row) to 300, m from 2 to 20, ragged tails.  The
    mixed path takes the instances with n >= 37: in the degenerate tiny ones (every
    grid point a landmark, gamma up to 1e10) the projected Hessian is beyond an FP32
    Cholesky, which the library reports per instance as NYS_ENOTSPD."""
    probs = ni.small_bvp(12)
    if precision == "mixed":
        probs = [q for q in probs if q["n"] >= 37]
    _check(api, probs, precision)


def test_paper_problems_11_to_13(api):
    """Tabulated singular coefficients (the table's t = 0 entry is never used);
    FP64 (the truncated landmark kernel, 9 of 20 eigenpairs, is refused by the
    mixed path)."""
    _check(api, [p for p, _ in paper_problems()], "fp64")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ivp_and_bvp_instances_in_one_batch(api, precision):
    """Initial and boundary value instances on the same landmark set (same n, m and
    h / sigma) share one factor; each keeps its own rows and condition rows."""
    probs = []
    for a, b in zip(ni.m0(3, n=2000), ni.bvp_family(3, n=2000)):
        probs += [a, b]
    _check(api, probs, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bvp_family_full_size_sample(api, precision):
    """The n = 1e4, m = 50 boundary value family (a few instances)."""
    _check(api, ni.bvp_family(4), precision)


def test_bvp_family_full_size_batch_sampled(api):
    """The 4096-instance boundary value batch in the configuration bench.py times
    (mixed, default refinement); sampled instances against the oracle."""
    import torch
    probs = ni.bvp_family(4096)
    bt = api.Batch(probs, precision="mixed")
    x, st = bt.run()
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    pick = [0, 1, 777, 2048, 4095]                  # increasing: queries in instance order
    grids = [core.grid(probs[k]) for k in pick]
    lens = np.zeros(4096, dtype=np.int64)
    for k, g in zip(pick, grids):
        lens[k] = len(g)
    off = torch.tensor(np.r_[0, np.cumsum(lens)], dtype=torch.int64, device="cuda")
    tq = torch.tensor(np.concatenate(grids), dtype=torch.float64, device="cuda")
    y, _ = bt.eval(tq, off)
    yc = y.cpu().numpy()
    pos = 0
    for k, g in zip(pick, grids):
        ref = core.solve_linear(probs[k])
        got = yc[pos:pos + len(g)]
        pos += len(g)
        assert np.abs(got - ref["y"]).max() <= TOL["mixed"] * np.abs(ref["y"]).max(), k
    bt.close()


def test_gradient_refuses_boundary_value_batches(api):
    import torch
    from paper_2510_04094_gb300 import _abi as A
    bt = api.Batch(ni.small_bvp(2), precision="fp64")
    bt.run()
    torch.cuda.synchronize()
    obs = [np.array([0.1]), np.array([0.2])]
    with pytest.raises(A.NysError) as e:
        bt.grad(obs, None, np.ones(2))
    assert e.value.code == A.NYS_EINVAL
    bt.close()


def test_update_cannot_switch_conditions(api):
    from paper_2510_04094_gb300 import _abi as A
    probs = ni.small_bvp(2)
    bt = api.Batch(probs, precision="fp64")
    flipped = [dict(q, bc="ivp") for q in probs]
    with pytest.raises(A.NysError) as e:
        bt.update(flipped)
    assert e.value.code == A.NYS_EINVAL
    bt.close()


def test_update_of_tabulated_coefficients(api):
    """An update that keeps every landmark set (same grid spacing and sigma) but
    changes the tabulated right-hand sides and boundary values."""
    import torch
    probs = [p for p, _ in paper_problems()]
    bt = api.Batch(probs, precision="fp64")
    bt.run()
    new = [dict(q, r=np.asarray(q["r"]) * 0.5 + 0.25, v=[q["v"][0] - 0.1, q["v"][1] + 0.2]) for q in probs]
    bt.update(new)
    bt.run()
    y, _ = bt.eval([core.grid(q) for q in new])
    torch.cuda.synchronize()
    assert (bt.status.cpu().numpy() == 0).all()
    yc = y.cpu().numpy()
    off = 0
    for q in new:
        ref = core.solve_linear(q)
        ref2 = core.solve_linear_nullspace(q)
        scale = np.abs(ref["y"]).max()
        tol = max(1e-10, 10 * np.abs(ref["y"] - ref2["y"]).max() / scale)
        assert np.abs(yc[off:off + q["n"]] - ref["y"]).max() <= tol * scale
        off += q["n"]
    bt.close()


# ---- nonlinear boundary value problems (nys_newton) --------------------------
def _nl_bvp(P, q, n=200, m=20, sigma=0.3, gamma=1e10, T=1.0, delta=0.0, g=0.0, w=0.0):
    return dict(p=2, n=n, m=m, t0=0.0, t1=T, sigma=sigma, gamma=gamma, v=list(q), kind="nl",
                P=list(P), delta=delta, g=g, omega=w, bc="bvp")


def _newton_compare(api, probs, max_iter=50, tol=1e-10, ytol=1e-10):
    """Same iteration counts and statuses as the oracle's Newton; fitted values and
    auxiliary unknowns (rows 2..n-1 for boundary values) to ytol."""
    import torch
    from oracle import newton
    bt = api.Batch(probs, precision="fp64")
    x, st, iters, yaux = bt.newton(max_iter=max_iter, tol=tol, want_y=True)
    grids = [core.grid(q) for q in probs]
    y, _ = bt.eval(grids)
    torch.cuda.synchronize()
    st, iters, y, yaux = st.cpu().numpy(), iters.cpu().numpy(), y.cpu().numpy(), yaux.cpu().numpy()
    bt.close()
    off = offy = 0
    for k, q in enumerate(probs):
        ref = newton.solve(q, tol=tol, max_iter=max_iter)
        n = q["n"]
        assert iters[k] == ref["iters"], (k, iters[k], ref["iters"])
        assert (st[k] == 0) == ref["converged"], (k, st[k])
        if ref["converged"]:
            ny = len(ref["y_aux"])
            err = np.abs(y[off:off + n] - ref["y"]).max() / np.abs(ref["y"]).max()
            erry = np.abs(yaux[offy:offy + ny] - ref["y_aux"]).max() / np.abs(ref["y_aux"]).max()
            assert err <= ytol and erry <= 10 * ytol, (k, err, erry)
        off += n
        offy += n - 1   # the device keeps n - 1 auxiliary unknowns per instance


def test_nonlinear_bvps_with_closed_forms(api):
    """y'' = 2 y^3 (y = 1/(1+t)) and y'' = y^2 (y = 6/(1+t)^2) on [0, 1]."""
    probs = [_nl_bvp([0.0, 0.0, 0.0, 2.0], (1.0, 0.5)), _nl_bvp([0.0, 0.0, 1.0, 0.0], (6.0, 1.5)),
             _nl_bvp([0.0, 0.0, 0.0, 2.0], (1.0, 0.5), n=2000, m=40, sigma=0.05)]
    _newton_compare(api, probs)


def test_nonlinear_bvp_and_ivp_instances_in_one_batch(api):
    """Duffing-type boundary value problems on [0, 2] beside initial value problems
    of the same kind (each with its own rows and conditions)."""
    rng = np.random.default_rng(5)
    probs = []
    for k in range(6):
        a, b = rng.uniform(0.2, 1.0), rng.uniform(0.5, 2.0)
        q = _nl_bvp([0.0, -a, 0.0, -b], tuple(rng.uniform(-0.5, 0.5, 2)), n=int(rng.integers(80, 400)),
                    m=int(rng.integers(8, 24)), T=2.0, delta=0.3, g=0.5, w=1.2, gamma=1e8)
        q["sigma"] = q["t1"] / q["m"] * 1.3
        if k % 2:
            q["bc"] = "ivp"
        probs.append(q)
    _newton_compare(api, probs)


# ---- right-hand side nonlinear in y' (beta y'^2 / y; Problem 15) ------------
def _p15(n=300, m=10, sigma=1.0, gamma=1e7, beta=2.0, c1=-1.0, bc="bvp"):
    """y'' = c1 y + beta (y')^2 / y on [-1, 1]; Appendix A.6 has c1 = -1, beta = 2,
    y(+-1) = 1 / (2 cosh 1).  The initial value version starts from the closed form."""
    q = 0.5 / np.cosh(1.0)
    v = [q, q] if bc == "bvp" else [q, 0.5 * np.sinh(1.0) / np.cosh(1.0) ** 2]
    return dict(p=2, n=n, m=m, t0=-1.0, t1=1.0, sigma=sigma, gamma=gamma, v=v, kind="nl",
                P=[0.0, c1, 0.0, 0.0], delta=0.0, beta=beta, g=0.0, omega=0.0, bc=bc)


def test_problem_15_on_the_gpu(api):
    """The paper's Problem 15 with its printed hyper-parameters: the oracle's
    iteration count and fit, and the printed accuracy against y = 1 / (2 cosh t)."""
    import torch
    prob = _p15()
    _newton_compare(api, [prob])
    bt = api.Batch([prob], precision="fp64")
    x, st, iters, _ = bt.newton()
    y, _ = bt.eval([core.grid(prob)])
    torch.cuda.synchronize()
    t = core.grid(prob)
    e = np.abs(y.cpu().numpy() - 0.5 / np.cosh(t))
    assert int(st.cpu().numpy()[0]) == 0
    assert e.mean() <= 2 * 1.68e-7 and e.max() <= 2 * 3.46e-7
    bt.close()


def test_beta_family_batch(api):
    """Variants of Problem 15 (beta, c1), its initial value form and a finer grid,
    beside a beta-free instance in one batch (two kinds of Newton rows)."""
    probs = [_p15(), _p15(beta=1.5, c1=-0.5, n=220, m=14, sigma=0.4, gamma=1e9),
             _p15(beta=2.5, c1=-1.5, n=180, m=12, sigma=0.5, gamma=1e8),
             _p15(bc="ivp", n=240, m=16, sigma=0.4, gamma=1e9),
             _p15(n=2000, m=20, sigma=0.3, gamma=1e10),
             _nl_bvp([0.0, 0.0, 0.0, 2.0], (1.0, 0.5))]
    _newton_compare(api, probs)
