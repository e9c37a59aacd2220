"""Host-side logic of bench.py: the FLOP counts its roofline divides and the
oracle baseline's process pool (no GPU needed)."""
import pytest

import nys_inputs as ni


@pytest.fixture(scope="module")
def bench():
    import bench as mod   # the repository root is on sys.path (conftest)
    return mod


def test_method_flop_count_per_row(bench):
    # 2m^2 + (m+1)(m+2) + 2(m+1) + 10m at the landmark counts of the workloads
    assert [bench.F_row(m) for m in (20, 32, 50, 64, 100)] == [1504, 3556, 8254, 13252, 31504]
    q = ni.m0(1)[0]
    assert bench.dense_flops([q]) == 9999 * 8254


def test_banded_and_issued_counts_are_consistent(bench):
    q = ni.m0(1)[0]
    useful = bench.banded_flops([q])
    issued = bench.tc_issued_flops([q])
    # every row sees about 22 landmarks of its band; the tensor-core kernel issues
    # more than the banded count (block packing, hi/lo products); on this family
    # every 256-row sub-chunk fits 16-slot blocks: 32 rows per 128 x 128 x 8 MMA
    assert 9999 * 400 < useful < 9999 * 800
    assert issued > useful
    assert issued == 40 * 2 * 4 * (2.0 * 128 * 128 * 8)   # 40 sub-chunks x 2 stages x 4 MMAs
    assert bench.dense_flops([q]) > useful


def test_oracle_baseline_pool_runs_single_threaded_workers(bench):
    probs = ni.m0(4, n=300, m=10)
    rate, done, wall = bench.oracle_baseline(probs, 0.01, 2)
    assert done >= 2 and rate > 0 and wall > 0
