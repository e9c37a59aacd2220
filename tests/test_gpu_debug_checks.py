"""The debug build (build(debug=True), NYS_DEBUG_CHECKS): its kernels check their
shared- and global-memory indices and report a failed check as NYS_EBOUNDS
instead of reading or writing out of bounds.  On valid batches no check may fail
and the results must equal the release build's bit for bit (the checks only
guard accesses).  The debug library runs in a child process (one library per
process); the batches cover the band kernels, the tensor-core windows, the
compact large-m eigendecomposition (odd m) and the FP64 path."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2510_04094_gb300.build as B
if sys.argv[2] == "debug":
    B.LIB_PATH = B.build(debug=True)
else:
    B.build()
import torch
from paper_2510_04094_gb300 import api
import nys_inputs as ni

def cap_batch():
    fam = ni.linear_family(6, n=1000, m=100, T=10.0, name="small", sub=31)
    shapes = [(140, 112), (130, 112), (700, 101), (400, 105), (3000, 112), (1000, 101)]
    return [dict(q, n=n, m=m, sigma=1.5 * (q["t1"] - q["t0"]) / (m - 1)) for q, (n, m) in zip(fam, shapes)]

out = {}
cases = [("m0", ni.m0(64, n=3000), "mixed"), ("ragged", ni.cfg3(40, n_hi=4000), "mixed"),
         ("cap", cap_batch(), "mixed"), ("ragged64", ni.cfg3(12, n_hi=3000), "fp64")]
for name, probs, prec in cases:
    bt = api.Batch(probs, precision=prec)
    bt.run()
    torch.cuda.synchronize()
    out[name] = {"status": bt.status.cpu().numpy().tolist(), "x": bt.x.cpu().numpy().tolist()}
    bt.close()
json.dump(out, open(sys.argv[3], "w"))
"""


def _run(kind, path):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, kind, path], capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.load(open(path))


def test_debug_build_checks_pass_and_match_release():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with tempfile.TemporaryDirectory() as d:
        rel = _run("release", os.path.join(d, "rel.json"))
        dbg = _run("debug", os.path.join(d, "dbg.json"))
    for name in rel:
        st = np.asarray(dbg[name]["status"])
        assert (st == 0).all(), (name, st)      # no NYS_EBOUNDS (-10), nothing else either
        assert (np.asarray(rel[name]["status"]) == 0).all(), name
        assert np.array_equal(np.asarray(rel[name]["x"]), np.asarray(dbg[name]["x"])), name
