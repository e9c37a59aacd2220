#!/usr/bin/env python
"""Throughput benchmark: batched Nystrom LS-SVM ODE solves on GB300.

Workload (default): 4096 instances of y'' + a y' + b y = c sin(omega t) on [0, 20],
n = 10^4 collocation points, m = 50 landmarks, sigma = 0.5, gamma = 1e10, seeded
synthetic coefficients (a ~ U[0,1], b ~ U[1,4], c ~ U[-1,1], omega ~ U[0.5,5],
y(0), y'(0) ~ N(0,1)).  One step = Nystrom setup + fused assembly + solve +
refinement for the whole batch (nys_run, one CUDA graph), inputs resident.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own batch
(weak scaling; no collective on the data path, one all-reduce for the timing).

Roofline (mixed path): the fused assembly of the metric workload runs on the band
kernel (FP32 FMAs on the CUDA cores); its rate counts the banded Gram each row
needs -- (a_i + 2)(a_i + 3) + 6 a_i FLOPs with a_i the landmarks within
u = ((t_i - s_j)/sigma)^2 <= 16 of row i -- and divides it by the measured FP32
FMA peak (include/nys_peak.h probes, run in the same process).  The method's
dense count per row, F(m) = 2m^2 (projection phi = W k) + (m+1)(m+2)
(upper-triangle Gram) + 2(m+1) (right-hand side) + 10m (operator), is reported
beside it as the method-equivalent rate; the FP64 path divides F(m) by the
measured DFMA peak.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched ODE solves/s at n=1e4, m=50"
UNIT = "solves/s"
LAG_U = 80.0   # kernel values exp(-u) with u > 80 (< 2e-35) are treated as zero
# DRAM bytes (read + write) of one k_assemble_band launch per instance of the
# metric family, from an ncu capture of the current kernel at 2048 instances
# (1285.9 KB + 5.6 KB; None once the kernel changes without a new capture).
# The unit Grams it writes stay in L2 during the launch.
BAND_DRAM_BYTES_PER_INSTANCE = (1285888 + 5632) / 2048


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--n", type=int, default=10_000)
    ap.add_argument("--m", type=int, default=50)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--assembly", default="auto", choices=["auto", "tc", "simt"],
                    help="MIXED assembly kernels (nys_assembly); the default is the library's")
    ap.add_argument("--workload", default="metric", choices=["metric", "ragged"],
                    help="ragged: the 4096-instance ragged family instead of the metric batch "
                         "(for launch lists and profiles)")
    ap.add_argument("--no-extras", action="store_true", help="skip the side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--long-time", action="store_true",
                    help="only time the long-time single instances (n = 5e4, m = 200) by phase")
    return ap.parse_args()


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, ws, local


def rank_problems(rank, B, n, m):
    """The batch of one rank (weak scaling: every rank solves its own B instances of
    the family, rank 0 the metric batch itself, rank r > 0 the family under spawn key r)."""
    import nys_inputs as ni
    return ni.linear_family(B, n=n, m=m, name="m0", sub=rank) if rank else ni.m0(B, n=n, m=m)


def job_rate(ms_local, B, ws, device=None):
    """Whole-job solves/s: every rank's B instances over the slowest rank's step time
    (one MAX all-reduce; the only collective of the job)."""
    import torch
    ms_t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if ws > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms = float(ms_t.item())
    return ws * B / (ms / 1000.0), ms


class Clocks:
    """nvidia-smi sampler (SM clock, max clock, throttle reasons) during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "power_w_max": max(pw), "samples": len(sm)}


# ---- FLOP counts ------------------------------------------------------------------
def F_row(m):
    """The method's FLOPs per collocation row: 2m^2 (projection) + (m+1)(m+2) (Gram,
    upper triangle, FMA = 2) + 2(m+1) (right-hand side) + 10m (operator)."""
    return 2 * m * m + (m + 1) * (m + 2) + 2 * (m + 1) + 10 * m


def rows_of(q):
    return q["n"] - 1 - (1 if q.get("bc") == "bvp" else 0)


def dense_flops(problems):
    return float(sum(rows_of(q) * F_row(q["m"]) for q in problems))


def _band(q, u=None):
    import numpy as np
    n, m = q["n"], q["m"]
    h = (q["t1"] - q["t0"]) / (n - 1)
    K = int(min(n - 1, math.ceil(math.sqrt(LAG_U if u is None else u) / (h / q["sigma"]))))
    j = np.arange(m)
    idx = (j * (n - 1) + (m - 1) // 2) // (m - 1)
    return idx, K


def banded_flops(problems, u=None):
    """FLOPs of the Gram over the landmarks inside each row's band (a_i of them,
    u = ((t_i - s_j)/sigma)^2 <= u, default the FP64 band LAG_U):
    (a_i + 2)(a_i + 3) + 6 a_i per row (exponentials on the SFU, not counted)."""
    import numpy as np
    cache, tot = {}, 0.0
    for q in problems:
        key = (q["n"], q["m"], q["t0"], q["t1"], q["sigma"], u)
        if key not in cache:
            idx, K = _band(q, u)
            i = np.arange(1, q["n"])
            a = (np.searchsorted(idx, i + K, side="right") - np.searchsorted(idx, i - K, side="left")).astype(float)
            cache[key] = float(np.sum((a + 2) * (a + 3) + 6 * a))
        tot += cache[key]
    return tot


BAND_U = 16.0         # the FP32 assembly Grams keep the landmarks with u <= 16
TC_BAND_U = BAND_U    # the tensor-core Gram's sub-chunk windows
TC_SUB_ROWS = 256
TC_MMA_STEPS = 8      # MMA steps per tensor-memory accumulator entry, at most


def slot_block(M2):
    return 16 if M2 <= 16 else (32 if M2 <= 32 else 64)


def tc_issued_flops(problems, num_sms=152):
    """TF32 MMA FLOPs k_assemble_tc issues for the batch.  Work units of
    max(256, rows / max(B, 4 SMs)) rows per instance are cut into sub-chunks of
    up to 256 rows; a sub-chunk whose landmark window (rows within u <= 16) has
    M2 = A + 2 columns uses slot blocks of Bs = 16, 32, 64 (M2 <= Bs) and 4 MMAs
    of 128 x 128 x 8 per stage of 2048 / Bs rows, or, for M2 > 64, 6 MMAs of
    128 x N x 8 (N = M2 rounded up to 16) per stage of 16 rows; sub-chunks are
    cut to 8 * 512 / Bs rows (32 when M2 > 64)."""
    import numpy as np
    total = sum(rows_of(q) for q in problems)
    target = max(len(problems), 4 * num_sms)
    upr = max(TC_SUB_ROWS, -(-total // target))
    cache, tot = {}, 0.0
    for q in problems:
        key = (q["n"], q["m"], q["t0"], q["t1"], q["sigma"], q.get("bc"))
        if key not in cache:
            idx, _ = _band(q)
            n, m = q["n"], q["m"]
            hs = (q["t1"] - q["t0"]) / (n - 1) / q["sigma"]
            Kb = int(min(math.ceil(math.sqrt(TC_BAND_U) / hs), n))
            nrows = rows_of(q)
            units = max(1, -(-nrows // upr))

            def window(a, b):
                return int(np.searchsorted(idx, b - 1 + Kb, side="right")
                           - np.searchsorted(idx, a - Kb, side="left"))
            f = 0.0
            for u in range(units):
                r0 = 1 + nrows * u // units
                r1 = 1 + nrows * (u + 1) // units
                s0 = r0
                while s0 < r1:
                    L = min(TC_SUB_ROWS, r1 - s0)
                    M2 = window(s0, s0 + L) + 2
                    cap = TC_MMA_STEPS * 512 // slot_block(M2) if M2 <= 64 else 32
                    if L > cap:        # at most TC_MMA_STEPS MMAs per accumulator entry
                        L = cap
                        M2 = window(s0, s0 + L) + 2
                    if M2 <= 64:
                        Bs = slot_block(M2)
                        f += -(-L // (2048 // Bs)) * 4 * 2.0 * 128 * 128 * 8
                    else:
                        N = -(-M2 // 16) * 16
                        f += -(-L // 16) * 6 * 2.0 * 128 * N * 8
                    s0 += L
            cache[key] = f
        tot += cache[key]
    return tot


def band_issued_flops(problems):
    """FP32 FMA FLOPs k_assemble_band issues: 136 FMAs (16 x 16 window Gram,
    upper triangle) per row of every window, rows past a unit's end included."""
    import numpy as np
    tot = 0.0
    for q in problems:
        tot += 2.0 * 136 * rows_of(q)
    return tot


# ---- CPU oracle baseline ---------------------------------------------------------------
def _oracle_worker(job):
    """Solve problems with the oracle (numpy FP64, one BLAS thread) for about
    `seconds`; returns (count, elapsed).  Runs in a spawned process."""
    probs, seconds = job
    from oracle import core
    t0 = time.perf_counter()
    k = 0
    for q in probs:
        core.solve_linear(q)
        k += 1
        if time.perf_counter() - t0 > seconds:
            break
    return k, time.perf_counter() - t0


def oracle_baseline(problems, seconds, workers):
    """Oracle solves/s on `workers` host cores (one single-threaded process per
    core, spawned), each solving its own slice of the batch for ~`seconds`.
    Returns (solves/s, solved, wall seconds)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            pool.map(_oracle_worker, [(problems[:1], 0.0)] * workers)   # imports, BLAS start-up
            per = max(1, len(problems) // workers)
            jobs = [(problems[w * per:(w + 1) * per] or problems[:per], seconds) for w in range(workers)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, jobs)
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    done = sum(r[0] for r in res)
    return done / wall, done, wall


def workload_config(args, ws):
    if args.workload == "ragged":
        return {"workload": "ragged linear 2nd-order ODE batch, n log-uniform in [500, 2e4], "
                            "m in {20,32,50,64,100}, sigma=T/m, gamma=1e10, %s" % args.precision,
                "global_batch": ws * args.batch, "parallelism": "dp%d" % ws,
                "l2": "flushed between steps (256 MB write)"}
    return {"workload": "linear 2nd-order ODE batch y''+ay'+by=c sin(wt), n=%d, m=%d, "
                        "sigma=0.5, gamma=1e10, %s" % (args.n, args.m, args.precision),
            "global_batch": ws * args.batch, "seq_len": args.n, "parallelism": "dp%d" % ws,
            "l2": "flushed between steps (256 MB write)"}


def run_reference(args, rank, ws):
    """The oracle (the paper ships no code) on the host cores, one process per core."""
    import nys_inputs as ni
    if rank != 0:
        return
    probs = ni.m0(args.batch, n=args.n, m=args.m)
    cores = os.cpu_count() or 1
    per_step = max(0.5, min(4.0, 60.0 / max(1, args.steps + args.warmup)))
    oracle_baseline(probs[:cores], 0.05, cores)                    # warm-up
    tot_k, tot_t = 0, 0.0
    for s in range(args.steps):
        rate, k, wall = oracle_baseline(probs, per_step, cores)
        tot_k += k
        tot_t += wall
    value = tot_k / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d instances of the workload, numpy FP64 oracle, %d "
                                       "single-threaded processes, %.1f s" % (tot_k, cores, tot_t)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---- GPU side measurements -------------------------------------------------------------
def ev_ms(fn, reps, stream, flush=None):
    """Mean ms of fn() over reps launches, CUDA events on `stream` (L2 flushed
    before each, outside the events)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ts) / reps


def measure_peaks(local):
    from paper_2510_04094_gb300 import peaks
    clk = Clocks(local).start()
    time.sleep(0.3)
    out = {k: peaks.measure(k) for k in ("tf32_mma", "bf16_mma", "ffma", "dfma")}
    out["clocks"] = clk.stop()
    return out


def long_time_breakdown(Batch, ni, torch):
    """Single long-time instances at the sizes of Table 12 (FP64): ms per nys_run
    (factor + assembly + solve, one graph; the factor overlaps the assembly on a
    side stream), per nys_assemble and per nys_solve, each the mean of 3 calls
    timed with CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()
    out = {}
    for nm in ("P3", "P9"):
        q, _ = ni.long_time(nm)
        bt = Batch([q], precision="fp64")
        res = {"n": q["n"], "m": q["m"], "run_ms": ev_ms(bt.run, 3, stream),
               "assemble_ms": ev_ms(bt.assemble, 3, stream), "solve_ms": ev_ms(bt.solve, 3, stream)}
        _, st = bt.solve()
        torch.cuda.synchronize()
        res["m_eff"] = int(bt.m_eff()[0])
        res["status_ok"] = bool((st.cpu().numpy() == 0).all())
        out[nm] = res
        bt.close()
    return out


def rel_err_sample(bt, probs, ks):
    """Max relative error of the fitted y of instances ks against the oracle."""
    import numpy as np
    import torch
    from oracle import core
    grids = [core.grid(probs[k]) for k in ks]
    lens = np.zeros(len(probs), dtype=np.int64)
    for k, g in zip(ks, grids):
        lens[k] = len(g)
    off = torch.tensor(np.r_[0, np.cumsum(lens)], dtype=torch.int64, device="cuda")
    tq = torch.tensor(np.concatenate(grids), dtype=torch.float64, device="cuda")
    y, _ = bt.eval(tq, off)
    yc = y.cpu().numpy()
    pos, errs = 0, []
    for k, g in zip(ks, grids):
        ref = core.solve_linear(probs[k])["y"]
        errs.append(float(np.abs(yc[pos:pos + len(g)] - ref).max() / np.abs(ref).max()))
        pos += len(g)
    return max(errs)


def side_measurements(args, probs, bt, value, ws, local, stream, flush, peaks_out):
    """Everything beside the metric line's own numbers (rank 0): accuracy, the plain
    FP64 path on the same batch, per-kernel rooflines, other workloads."""
    import numpy as np
    import torch
    import nys_inputs as ni
    from paper_2510_04094_gb300.api import Batch

    ex = {}
    pk = peaks_out
    dfma, ffma = pk["dfma"]["tflops"], pk["ffma"]["tflops"]
    B = len(probs)
    ex["rel_err_vs_oracle_max"] = rel_err_sample(bt, probs, [0, 1, 777, 2048, B - 1] if B > 2048 else [0, B - 1])
    ex["status_ok"] = bool((bt.status.cpu().numpy() == 0).all())

    # refinement: one full pass (a solve with refine_steps = 1 minus a solve
    # without refinement, both after the same assembly) and the default's
    # adaptive pass (the default solve minus the one-pass solve)
    b0 = Batch(probs, precision=args.precision, refine_steps=0)
    b0.assemble()
    solve0 = ev_ms(b0.solve, 5, stream, flush)
    b0.close()
    solve_d = ev_ms(bt.solve, 5, stream, flush)
    ref_fl = float(sum(rows_of(q) * 4 * q["m"] for q in probs))
    ex["solve_ms"] = {"k_solve": solve0, "k_solve_plus_default_refinement": solve_d}
    rows = {}
    if args.precision == "mixed":
        b1 = Batch(probs, precision=args.precision, refine_steps=1)
        b1.assemble()
        solve1 = ev_ms(b1.solve, 5, stream, flush)
        b1.close()
        ex["solve_ms"]["k_solve_plus_one_pass"] = solve1
        t = max(1e-6, solve1 - solve0)
        ach = ref_fl / (t * 1e-3) / 1e12
        rows["refinement_pass"] = {
            "kernels": "k_refine_band (k_refine_rows for unplanned instances) + k_refine_update",
            "ms": t,
            "flop_count": "4m per row (residual and its projection), FP64-accurate (float-float)",
            "achieved_tflops": ach, "frac_of_dfma": ach / dfma, "frac_of_ffma": ach / ffma,
            "adaptive_pass_ms": solve_d - solve1}

    # the precision split: the same batch with the FP64 H and Cholesky factor
    if args.precision == "mixed":
        bf = Batch(probs, precision="mixed-f64f")
        msf = ev_ms(bf.run, 3, stream, flush)
        _, stf = bf.run()
        torch.cuda.synchronize()
        ex["mixed_fp64_factor"] = {
            "ms_per_step": msf, "solves_s": B / (msf * 1e-3),
            "fp32_factor_ms_per_step": B / value * 1e3 * ws,
            "rel_err_vs_oracle_max": rel_err_sample(bf, probs, [0, 1, 777, 2048, B - 1] if B > 2048 else [0, B - 1]),
            "status_ok": bool((stf.cpu().numpy() == 0).all())}
        bf.close()

    # the plain FP64 path on the same batch: batched (one graph) and per instance
    b64 = Batch(probs, precision="fp64")
    ms64 = ev_ms(b64.run, 3, stream, flush)
    asm64 = ev_ms(b64.assemble, 3, stream, flush)
    _, st64 = b64.run()
    torch.cuda.synchronize()
    fp64_err = rel_err_sample(b64, probs, [0, B - 1])
    b64.close()
    fl = dense_flops(probs)
    exec64 = float(sum(rows_of(q) * ((q["m"] + 2) * (q["m"] + 3) + 12 * q["m"]) for q in probs))
    rows["k_assemble_f64"] = {
        "ms": asm64, "achieved_tflops": fl / (asm64 * 1e-3) / 1e12,
        "peak_tflops": dfma, "frac": fl / (asm64 * 1e-3) / 1e12 / dfma,
        "issued_tflops": exec64 / (asm64 * 1e-3) / 1e12,
        "pipe_frac": exec64 / (asm64 * 1e-3) / 1e12 / dfma,
        "flop_count": "F(m) per row; issued: (m+2)(m+3) Gram + 12m operator per row"}
    single = Batch(probs[:1], precision="fp64")
    from paper_2510_04094_gb300 import _abi
    from paper_2510_04094_gb300.api import pack_instances, _stream_handle
    packed = [pack_instances([q]) for q in probs]
    single.run()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for arr, _keep in packed:                   # each instance by its own launch sequence
        _abi.nys_update(single.ctx, arr, _stream_handle())
        single.run()
    b.record(stream)
    torch.cuda.synchronize()
    ms_pi = a.elapsed_time(b)
    single.close()
    ex["fp64_path"] = {
        "instances": B, "timing": "CUDA events on the launching stream",
        "batched": {"ms_per_step": ms64, "solves_s": B / (ms64 * 1e-3),
                    "status_ok": bool((st64.cpu().numpy() == 0).all()), "rel_err_vs_oracle_max": fp64_err},
        "per_instance": {"ms_total": ms_pi, "solves_s": B / (ms_pi * 1e-3),
                         "how": "one single-instance context; per instance nys_update + nys_run"}}
    ex["speedup_vs_fp64_batched"] = value / ws / ex["fp64_path"]["batched"]["solves_s"]
    ex["speedup_vs_fp64_per_instance"] = value / ws / ex["fp64_path"]["per_instance"]["solves_s"]

    # adjoint gradient (nys_grad): 1024 instances, n = 5000, m = 50, 200 observations, FP64
    g4, tau4, yobs4 = ni.cfg4()
    bg = Batch(g4, precision="fp64")
    tq, tq_off = bg._queries(list(tau4), None)
    bg.run()
    yq, _ = bg.eval(tq, tq_off)
    u = 2.0 * (yq - torch.tensor(np.concatenate(yobs4), device=yq.device)) / tau4.shape[1]
    gms = ev_ms(lambda: bg.grad(tq, tq_off, u), 5, stream, flush)
    gfl = float(sum(rows_of(q) * 12 * q["m"] for q in g4))
    rows["nys_grad"] = {"instances": len(g4), "ms": gms,
                        "flop_count": "12m per row (adjoint row pass)",
                        "achieved_tflops": gfl / (gms * 1e-3) / 1e12,
                        "frac_of_dfma": gfl / (gms * 1e-3) / 1e12 / dfma,
                        "fp64_solve_ms": ev_ms(bg.run, 3, stream, flush)}
    bg.close()

    # batched Newton family: 64 logistic / Duffing instances, n in [2000, 1e4], FP64, cap 20
    b5 = Batch(ni.cfg5(), precision="fp64")
    ms5 = ev_ms(lambda: b5.newton(max_iter=20, tol=1e-10), 2, stream)
    _, st5, it5, _ = b5.newton(max_iter=20, tol=1e-10)
    its = it5.cpu().numpy()
    nfl = float(sum(rows_of(q) * (4 * q["m"] ** 2 + 3 * (q["m"] + 1) ** 2) * (int(k) + 1)
                    for q, k in zip(b5.problems, its)))
    rows["nys_newton"] = {"instances": len(b5.problems), "ms": ms5,
                          "iterations_max": int(its.max()), "converged": int((st5 == 0).sum().item()),
                          "flop_count": "(4m^2 + 3(m+1)^2) per row and row pass (iterations + 1 passes)",
                          "achieved_tflops": nfl / (ms5 * 1e-3) / 1e12,
                          "frac_of_dfma": nfl / (ms5 * 1e-3) / 1e12 / dfma}
    b5.close()
    ex["rooflines"] = rows

    # ragged batched family: 4096 instances, n log-uniform in [500, 2e4], m in
    # {20, 32, 50, 64, 100}, sigma = T/m, one CUDA graph per step
    r3 = Batch(ni.cfg3(), precision="mixed")
    ms3 = ev_ms(r3.run, 3, stream, flush)
    ex["ragged_4096"] = {"ms_per_step": ms3, "solves_s": len(r3.problems) / (ms3 / 1000.0),
                         "rows": int(sum(q["n"] - 1 for q in r3.problems))}
    r3.close()
    # boundary value family (Appendix A.4): 4096 x (n = 1e4, m = 50), mixed, default
    # refinement for boundary values (two passes)
    pb = ni.bvp_family(4096)
    rb = Batch(pb, precision="mixed")
    msb = ev_ms(rb.run, 3, stream, flush)
    ex["bvp_4096"] = {"ms_per_step": msb, "solves_s": 4096 / (msb / 1000.0), "refine_passes": 2,
                      "rel_err_vs_oracle_max": rel_err_sample(rb, pb, [0, 1, 4095]),
                      "status_ok": bool((rb.status.cpu().numpy() == 0).all())}
    rb.close()
    single = {}
    for prec in ("fp64", "mixed"):
        s1 = Batch([ni.cfg2_linear()], precision=prec)
        single["linear_" + prec + "_ms"] = ev_ms(s1.run, 3, stream)
        s1.close()
    sn = Batch([ni.cfg2_tanh()], precision="fp64")
    single["tanh_newton_ms"] = ev_ms(lambda: sn.newton(max_iter=50, tol=1e-10), 2, stream)
    sn.close()
    ex["single_n1e4"] = single
    try:
        ex["long_time_n5e4_m200"] = long_time_breakdown(Batch, ni, torch)
    except Exception as e:   # a side measurement must not cost the metric line
        ex["long_time_n5e4_m200"] = {"error": repr(e)[:200]}
    try:
        hp = ni.small_higher(1024, sub=7, n_choices=(1000, 2000), m_choices=(20, 32))
        bh = Batch(hp, precision="fp64")
        msh = ev_ms(bh.run, 3, stream, flush)
        _, sth = bh.run()
        torch.cuda.synchronize()
        ex["higher_order_1024"] = {"ms_per_step": msh, "solves_s": len(hp) / (msh / 1000.0),
                                   "status_ok": bool((sth.cpu().numpy() == 0).all())}
        bh.close()
    except Exception as e:
        ex["higher_order_1024"] = {"error": repr(e)[:200]}
    return ex


def main():
    args = parse()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import nys_inputs as ni
    from paper_2510_04094_gb300 import _abi
    from paper_2510_04094_gb300.api import Batch, pack_instances, _stream_handle

    if args.long_time:
        if rank == 0:
            print(json.dumps({"workload": "long-time single instances, Table 12 sizes, FP64",
                              "unit": "ms", "data": "synthetic",
                              "results": long_time_breakdown(Batch, ni, torch)}))
        return

    B = args.batch
    probs = (rank_problems(rank, B, args.n, args.m) if args.workload == "metric"
             else ni.cfg3(B))
    bt = Batch(probs, precision=args.precision, assembly=args.assembly)
    # default refinement: one pass and the adaptive pass (launched for every
    # batch; instances already converged skip it)
    refine = 2 if args.precision == "mixed" else 0
    # setup (lag tables, eigendecomposition, condition rows), assembly, solve, 2 per
    # refinement pass (the band or row residual pass and the update)
    launches_per_step = 3 + 2 + 2 * refine
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(3, args.warmup)):
        bt.run()
    torch.cuda.synchronize()
    clocks = Clocks(local).start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()                      # evict L2 between steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.run()
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in times) / args.steps
    value, ms = job_rate(ms, B, ws, device="cuda")

    # dominant kernel (fused assembly) on the launching stream
    asm_ms = ev_ms(bt.assemble, max(3, args.steps), stream, flush)
    bt.solve()
    torch.cuda.synchronize()

    # end to end through the public API: host instances -> H2D -> run -> D2H of x
    x_host = torch.empty_like(bt.x, device="cpu").pin_memory()
    arr_next, keep = pack_instances(
        ni.linear_family(B, n=args.n, m=args.m, name="m0", sub=100 + rank) if args.workload == "metric"
        else probs)
    arr_same, keep2 = pack_instances(probs)
    e2e_t = []
    for s in range(args.steps):
        arr = arr_next if s % 2 == 0 else arr_same
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _abi.nys_update(bt.ctx, arr, _stream_handle())
        bt.run()
        x_host.copy_(bt.x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t)
    h2d = int(_abi.nys_upload_bytes(bt.ctx))
    d2h = bt.x.numel() * 8
    _abi.nys_update(bt.ctx, arr_same, _stream_handle())
    bt.run()
    torch.cuda.synchronize()

    roof, extra, cpu_base = None, {}, None
    if rank == 0:
        pk = measure_peaks(local)
        fl = dense_flops(probs)
        method_rate = fl / (asm_ms * 1e-3) / 1e12
        mixed = args.precision == "mixed"
        band_items, other_items = bt.assembly_items() if mixed else (0, 1)
        if mixed and other_items == 0:
            # the band kernel: FP32 FMAs on the CUDA cores; its algorithmic work is
            # the banded Gram of every row (landmarks within u <= 16 of the row)
            bfl = banded_flops(probs, u=BAND_U)
            peak = pk["ffma"]["tflops"]
            roof = {"bound": "alu", "kernel": "k_assemble_band",
                    "achieved": bfl / (asm_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": bfl / (asm_ms * 1e-3) / 1e12 / peak,
                    "peak_source": "measured in this run: FFMA probe, burst",
                    "flop_count": "banded Gram per collocation row, (a_i+2)(a_i+3) + 6 a_i with a_i "
                                  "the landmarks within u = ((t_i - s_j)/sigma)^2 <= 16 of row i",
                    "flops_per_launch": bfl, "ms_per_launch": asm_ms,
                    "traffic": (BAND_DRAM_BYTES_PER_INSTANCE * B if BAND_DRAM_BYTES_PER_INSTANCE
                                and args.n == 10_000 and args.m == 50 else None),
                    "issued_fma_tflops": band_issued_flops(probs) / (asm_ms * 1e-3) / 1e12,
                    "method_equivalent": {
                        "flop_count": "F(m) = 2m^2+(m+1)(m+2)+2(m+1)+10m per collocation row",
                        "tflops": method_rate,
                        "vs_tf32_tensor_peak": method_rate / pk["tf32_mma"]["tflops"]}}
        else:
            peak = pk["tf32_mma"]["tflops"] if mixed else pk["dfma"]["tflops"]
            roof = {"bound": "tensor" if mixed else "alu",
                    "kernel": ("k_assemble_tc" + (" + k_assemble_band" if band_items else "")) if mixed
                              else "k_assemble_f64",
                    "achieved": method_rate, "peak": peak, "unit": "TFLOP/s", "frac": method_rate / peak,
                    "peak_source": ("measured in this run: tcgen05 kind::tf32 probe, burst" if mixed
                                    else "measured in this run: DFMA probe, burst"),
                    "flop_count": "F(m) = 2m^2+(m+1)(m+2)+2(m+1)+10m per collocation row",
                    "flops_per_launch": fl, "ms_per_launch": asm_ms, "traffic": None}
            if mixed:
                iss = tc_issued_flops(probs)
                roof["issued_tflops"] = iss / (asm_ms * 1e-3) / 1e12
                roof["pipe_frac"] = roof["issued_tflops"] / peak
                roof["banded_useful_tflops"] = banded_flops(probs) / (asm_ms * 1e-3) / 1e12
        extra["peaks"] = pk
        if not args.no_extras:
            extra.update(side_measurements(args, probs, bt, value, ws, local, stream, flush, pk))
            cores = os.cpu_count() or 1
            r1, k1, w1 = oracle_baseline(probs, args.cpu_seconds, 1)
            rN, kN, wN = oracle_baseline(probs, args.cpu_seconds, cores)
            cpu_base = {"value": rN, "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": "%d instances of the workload on %d single-threaded processes "
                                  "(one per host core), numpy FP64 oracle, %.1f s" % (kN, cores, wN),
                        "single_core": {"value": r1, "threads": 1,
                                        "sample": "%d instances, one process, one BLAS thread, %.1f s"
                                                  % (k1, w1)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": workload_config(args, ws),
            "e2e": {"value": ws * B / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "cpu_baseline": cpu_base,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    bt.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
