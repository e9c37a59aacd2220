"""GPU parity for landmark counts above the shared-memory kernels' 112 (up to 224):
the factor and the KKT solve in a global workspace, the Gram assembled in entry
parts and its row chunks summed by a many-CTA pass.  FP64 (the only precision
these counts take); tolerances as in the other FP64 parity tests: 1e-10 relative,
or 10x the oracle's own rounding spread where the problem is that sensitive (the
truncated, ill-conditioned landmark kernels of the long-time workloads)."""
import numpy as np
import pytest

import nys_inputs as ni
from oracle import core

from parity_helpers import check_fp64, tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_04094_gb300 import api as A
    return A


def test_ragged_large_landmark_batch(api):
    """m from 113 to 224, n from 300 to 3000, orders 1, 2 and 4, initial and
    boundary values, constant and tabulated coefficients."""
    check_fp64(api, ni.big_m(6))


def test_large_and_small_landmark_counts_in_one_batch(api):
    """Instances of both kinds of kernel in one batch: each solved by its own."""
    probs = ni.big_m(3, sub=1) + ni.small_linear(4) + ni.small_higher(2, sub=5) + ni.small_bvp(2, sub=6)
    check_fp64(api, probs)


@pytest.mark.parametrize("name", ["P3", "P8", "P9"])
def test_long_time_workloads(api, name):
    """Full-size long-time instances (n = 2e4 - 5e4, m = 200, gamma = 1e7, the sizes
    of Table 12): parity on every grid point, and the fit's error against the closed
    form of the oracle's order.  Problem 3 (sigma^2 = 10: 111 of 200 eigenpairs
    kept, omega coordinates) is that ill-conditioned: the oracle's own routes differ
    by 8e-6 there, and its closed-form error moves by 2x between machines."""
    q, exact = ni.long_time(name)
    (y,) = check_fp64(api, [q])
    t = core.grid(q)
    ref = core.solve_linear(q)
    e_gpu = np.abs(y - exact(t)).max()
    e_ora = np.abs(ref["y"] - exact(t)).max()
    assert e_gpu <= 2 * e_ora + 1e-9, (e_gpu, e_ora)


def test_large_landmark_update(api):
    """nys_update with new coefficients on the same landmark sets re-solves the
    large instances from their kept factor."""
    import torch
    probs = ni.big_m(2, sub=2)
    bt = api.Batch(probs, precision="fp64")
    bt.run()
    new = [dict(q) for q in probs]
    for q in new:
        if q["kind"] == "lin":
            q["c"] = -0.5 * q["c"] + 0.25
        else:
            q["r"] = 0.5 * np.asarray(q["r"]) + 0.1
    bt.update(new)
    x, st = bt.run()
    grids = [core.grid(q) for q in new]
    y, _ = bt.eval(grids)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    yc = y.cpu().numpy()
    off = 0
    for q, g in zip(new, grids):
        tol, scale, ref, _, _ = tolerance(q, g)
        assert np.abs(yc[off:off + len(g)] - ref["y"]).max() / scale <= tol
        off += len(g)
    bt.close()
