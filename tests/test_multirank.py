"""The multi-rank (torchrun) path of bench.py on CPU with gloo, world size 2:
per-rank batches are disjoint draws of the family, and the job rate uses the
slowest rank's step time (MAX all-reduce, the job's only collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    probs = bench.rank_problems(rank, 6, n=400, m=12)
    ms_local = 10.0 + 5.0 * rank            # rank 1 is the slower one
    rate, ms = bench.job_rate(ms_local, 6, ws)
    out[rank] = (rate, ms, [q["v"][0] for q in probs], [q["a"][0] for q in probs])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_rate_and_disjoint_batches():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        rate, ms, _, _ = res[rank]
        assert ms == pytest.approx(15.0)                      # the slower rank's time
        assert rate == pytest.approx(2 * 6 / 0.015)            # all instances of the job
    # rank 0 solves the metric batch itself, rank 1 an independent draw
    assert not np.allclose(res[0][2], res[1][2])
    assert not np.allclose(res[0][3], res[1][3])


def test_single_rank_rate_needs_no_process_group():
    import bench
    rate, ms = bench.job_rate(20.0, 4096, 1)
    assert ms == 20.0 and rate == pytest.approx(4096 / 0.02)
