"""The seeded workloads: their closed forms solve their ODEs (so accuracy figures
quoted against them mean what they say), and the ragged families span the cases
their docstrings promise."""
import numpy as np
import pytest

import nys_inputs as ni


def _lin_residual(q, y, t):
    """y^(p) + a_1 y^(p-1) [+ a_2 y] - c sin(omega t + phi0) by central differences."""
    h = 1e-3
    d = [y(t)]
    d.append((y(t + h) - y(t - h)) / (2 * h))
    d.append((y(t + h) - 2 * y(t) + y(t - h)) / h ** 2)
    p, a = q["p"], q["a"]
    lhs = d[p] + a[0] * d[p - 1] + (a[1] * d[0] if p == 2 else 0.0)
    return lhs - q["c"] * np.sin(q["omega"] * t + q["phi0"])


@pytest.mark.parametrize("name", ["P3", "P7", "P8", "P9"])
def test_long_time_closed_forms_solve_their_odes(name):
    q, y = ni.long_time(name)
    t = np.linspace(q["t0"] + 0.01, q["t1"] - 0.01, 4001)
    res = _lin_residual(q, y, t)
    scale = 1.0 + abs(q["a"][0]) + (abs(q["a"][1]) if q["p"] == 2 else 0.0)
    assert np.abs(res).max() <= 1e-4 * scale * (1 + q["c"])
    # initial values: y(0), and y'(0) for p = 2
    assert abs(y(np.array([q["t0"]]))[0] - q["v"][0]) <= 1e-12
    if q["p"] == 2:
        h = 1e-6
        yp = (y(np.array([q["t0"] + h])) - y(np.array([q["t0"] - h])))[0] / (2 * h)
        assert abs(yp - q["v"][1]) <= 1e-6


def test_big_m_family_spans_its_cases():
    probs = ni.big_m(24)
    assert all(112 < q["m"] <= 224 and q["m"] <= q["n"] for q in probs)
    assert {q["p"] for q in probs} == {1, 2, 4}
    assert {q["kind"] for q in probs} == {"lin", "table"}
    assert {q.get("bc", "ivp") for q in probs} == {"ivp", "bvp"}
    assert all(q["bc"] == "ivp" or q["p"] in (2, 4) for q in probs)


def test_higher_order_family_spans_its_cases():
    probs = ni.small_higher(32)
    assert {q["p"] for q in probs} == {3, 4}
    assert any(q["bc"] == "bvp" for q in probs) and all(q["bc"] == "ivp" or q["p"] == 4 for q in probs)
    for q in probs:
        assert np.shape(q["f"]) == (q["p"], q["n"]) and np.shape(q["r"]) == (q["n"],)


def test_generators_are_seeded():
    a, b = ni.big_m(3, sub=4), ni.big_m(3, sub=4)
    assert [q["n"] for q in a] == [q["n"] for q in b]
    assert all(np.array_equal(np.asarray(x.get("r", 0)), np.asarray(y.get("r", 0))) for x, y in zip(a, b))
