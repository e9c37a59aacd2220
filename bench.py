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
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz
# DRAM bytes (read + write) of one k_assemble_tc launch per instance, from an ncu
# capture of 304 instances of this workload (dram__bytes_read.sum 285.4 KB +
# dram__bytes_write.sum 0.3 KB); the kernel keeps its operands on chip, its HBM
# traffic is work descriptors and landmark indices only
TC_DRAM_BYTES_PER_INSTANCE = (285.44e3 + 0.256e3) / 304


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
    ap.add_argument("--no-extras", action="store_true", help="skip FP64/oracle side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
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
    """nvidia-smi sampler (SM clock, max clock, throttle reasons) during the timed region."""
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


LAG_U = 80.0   # kernel values exp(-u) with u > 80 (< 2e-35) are treated as zero


def _band_counts(q):
    """Per collocation row i = 1..n-1: number of landmarks j with |i - idx_j| <= K,
    K = min(n - 1, ceil(sqrt(80) sigma / h)) (the band of the RBF features)."""
    import numpy as np
    n, m = q["n"], q["m"]
    h = (q["t1"] - q["t0"]) / (n - 1)
    K = int(min(n - 1, math.ceil(math.sqrt(LAG_U) / (h / q["sigma"]))))
    j = np.arange(m)
    idx = (j * (n - 1) + (m - 1) // 2) // (m - 1)
    i = np.arange(1, n)
    return np.searchsorted(idx, i + K, side="right") - np.searchsorted(idx, i - K, side="left")


def asm_flops(problems):
    """Algorithmic FLOPs of one fused assembly pass over the banded features: per
    row, with a_i landmarks inside the band, (a_i + 2)(a_i + 3) for the upper
    triangle of the augmented Gram (FMA = 2) + 6 a_i for the feature polynomials
    (exponentials run on the SFU and are not counted)."""
    import numpy as np
    cache, tot = {}, 0
    for q in problems:
        key = (q["n"], q["m"], q["t0"], q["t1"], q["sigma"])
        if key not in cache:
            a = _band_counts(q).astype(float)
            cache[key] = float(np.sum((a + 2) * (a + 3) + 6 * a))
        tot += cache[key]
    return tot


def dense_flops(problems):
    """The dense minimum form of the method per row, 2m^2 (projection) + (m+1)(m+2)
    (Gram) + 2(m+1) (right-hand side) + 10m (operator), counted without the band."""
    return sum((q["n"] - 1) * (2 * q["m"] ** 2 + (q["m"] + 1) * (q["m"] + 2) + 2 * (q["m"] + 1)
                               + 10 * q["m"]) for q in problems)


def oracle_rate(problems, seconds):
    """Oracle solves/s on a bounded sample (the oracle as it stands, numpy FP64)."""
    from oracle import core
    t0 = time.perf_counter()
    k = 0
    while k < len(problems):
        core.solve_linear(problems[k])
        k += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return k / dt, k, dt


def workload_config(args, ws):
    """The workload both arms report (the reference arm times the oracle on a
    bounded sample of this same batch)."""
    return {"workload": "linear 2nd-order ODE batch y''+ay'+by=c sin(wt), n=%d, m=%d, "
                        "sigma=0.5, gamma=1e10, %s" % (args.n, args.m, args.precision),
            "global_batch": ws * args.batch, "seq_len": args.n, "parallelism": "dp%d" % ws,
            "l2": "flushed between steps (256 MB write)"}


def run_reference(args, rank, ws):
    import nys_inputs as ni
    if rank != 0:
        return
    probs = ni.m0(args.batch, n=args.n, m=args.m)
    per_step = max(0.5, min(4.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(probs[:2], per_step / 4)
    rates, tot_k, tot_t = [], 0, 0.0
    for s in range(args.steps):
        r, k, dt = oracle_rate(probs[s * 3:], per_step)
        rates.append(r)
        tot_k += k
        tot_t += dt
    value = tot_k / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d instances of the workload, %.1f s" % (tot_k, tot_t)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def long_time_breakdown(Batch, ni, torch):
    """Single long-time instances at the sizes of Table 12 (FP64): ms per nys_run
    (factor + assembly + solve, one graph; the factor overlaps the assembly on a
    side stream), per nys_assemble and per nys_solve, each the mean of 3 calls
    timed with CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()

    def ev_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    for nm in ("P3", "P9"):
        q, _ = ni.long_time(nm)
        bt = Batch([q], precision="fp64")
        res = {"n": q["n"], "m": q["m"], "run_ms": ev_ms(bt.run), "assemble_ms": ev_ms(bt.assemble),
               "solve_ms": ev_ms(bt.solve)}
        _, st = bt.solve()
        torch.cuda.synchronize()
        res["m_eff"] = int(bt.m_eff()[0])
        res["status_ok"] = bool((st.cpu().numpy() == 0).all())
        out[nm] = res
        bt.close()
    return out


def main():
    args = parse()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import nys_inputs as ni
    from paper_2510_04094_gb300 import _abi
    from paper_2510_04094_gb300.api import Batch, pack_instances

    if args.long_time:
        if rank == 0:
            print(json.dumps({"workload": "long-time single instances, Table 12 sizes, FP64",
                              "unit": "ms", "data": "synthetic",
                              "results": long_time_breakdown(Batch, ni, torch)}))
        return

    B = args.batch
    probs = rank_problems(rank, B, args.n, args.m)
    bt = Batch(probs, precision=args.precision)
    refine = 1 if args.precision == "mixed" else 0   # default refinement passes
    # setup (lag tables [mixed] + eigendecomposition), assembly, solve, 2 per refinement pass
    launches_per_step = (2 if args.precision == "mixed" else 1) + 2 + 2 * refine
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(3, args.warmup)):
        bt.run()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
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

    # dominant-kernel timing (fused assembly) on the launching stream
    asm_ms = []
    for _ in range(max(3, args.steps)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.assemble()
        e1.record(stream)
        asm_ms.append((e0, e1))
    torch.cuda.synchronize()
    asm_ms = sum(a.elapsed_time(b) for a, b in asm_ms) / len(asm_ms)
    bt.solve()
    torch.cuda.synchronize()
    fl = asm_flops(probs)
    achieved = fl / (asm_ms / 1000.0) / 1e12

    # end to end through the public API: host instances -> H2D -> run -> D2H of x
    x_host = torch.empty_like(bt.x, device="cpu").pin_memory()
    arr_next, keep = pack_instances(ni.linear_family(B, n=args.n, m=args.m, name="m0", sub=100 + rank))
    arr_same, keep2 = pack_instances(probs)
    e2e_t = []
    for s in range(args.steps):
        arr = arr_next if s % 2 == 0 else arr_same
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _abi.nys_update(bt.ctx, arr, C_stream(stream))
        bt.run()
        x_host.copy_(bt.x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t)
    h2d = int(_abi.nys_upload_bytes(bt.ctx))
    d2h = bt.x.numel() * 8
    _abi.nys_update(bt.ctx, arr_same, C_stream(stream))
    bt.run()
    torch.cuda.synchronize()

    extra = {}
    cpu_base = None
    if rank == 0 and not args.no_extras:
        from oracle import core
        # accuracy of the timed configuration against the FP64 oracle (sampled instances)
        k = 6
        grids = [core.grid(q) for q in probs[:k]]
        y, _ = bt.eval(grids)
        yc = y.cpu().numpy()
        off, errs = 0, []
        for q, g in zip(probs[:k], grids):
            ref = core.solve_linear(q)["y"]
            errs.append(float(np.abs(yc[off:off + len(g)] - ref).max() / np.abs(ref).max()))
            off += len(g)
        extra["rel_err_vs_oracle_max"] = max(errs)
        extra["status_ok"] = bool((bt.status.cpu().numpy() == 0).all())
        # plain FP64 path: batched and one instance per launch sequence
        sub = probs[:256]
        b64 = Batch(sub, precision="fp64")
        b64.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            b64.run()
        torch.cuda.synchronize()
        extra["fp64_batched_solves_s"] = 2 * len(sub) / (time.perf_counter() - t0)
        b64.close()
        singles = [Batch([q], precision="fp64") for q in probs[:16]]
        for sb in singles:
            sb.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sb in singles:
            sb.run()
        torch.cuda.synchronize()
        extra["fp64_per_instance_solves_s"] = len(singles) / (time.perf_counter() - t0)
        for sb in singles:
            sb.close()
        extra["speedup_vs_fp64_per_instance"] = value / ws / extra["fp64_per_instance_solves_s"]
        extra["asm_ms"] = asm_ms
        extra["asm_dense_equiv_tflops"] = dense_flops(probs) / (asm_ms / 1000.0) / 1e12
        # adjoint gradient (nys_grad) on the parameter-estimation workload:
        # 1024 instances, n = 5000, m = 50, 200 observations each, FP64
        g4, tau4, yobs4 = ni.cfg4()
        bg = Batch(g4, precision="fp64")
        tq, tq_off = bg._queries(list(tau4), None)
        bg.run()
        yq, _ = bg.eval(tq, tq_off)
        u = 2.0 * (yq - torch.tensor(np.concatenate(yobs4), device=yq.device)) / tau4.shape[1]
        for _ in range(3):
            bg.grad(tq, tq_off, u)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bg.run()
        e1.record(stream)
        for _ in range(5):
            bg.grad(tq, tq_off, u)
        e2.record(stream)
        torch.cuda.synchronize()
        extra["grad_cfg4"] = {"instances": len(g4), "fp64_solve_ms": e0.elapsed_time(e1),
                              "grad_ms": e1.elapsed_time(e2) / 5}
        bg.close()

        def step_ms(batch, fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b2 = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b2.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b2) / reps

        # ragged batched family: 4096 instances, n log-uniform in [500, 2e4],
        # m in {20, 32, 50, 64, 100}, sigma = T/m, one CUDA graph per step
        r3 = Batch(ni.cfg3(), precision="mixed")
        ms3 = step_ms(r3, r3.run)
        extra["ragged_4096"] = {"ms_per_step": ms3, "solves_s": len(r3.problems) / (ms3 / 1000.0),
                                "rows": int(sum(q["n"] - 1 for q in r3.problems))}
        r3.close()
        # boundary value family (Appendix A.4): 4096 x (n = 1e4, m = 50), mixed, the
        # library's default refinement for boundary values (two passes); error of a
        # few instances against the FP64 oracle
        rb = Batch(ni.bvp_family(4096), precision="mixed")
        msb = step_ms(rb, rb.run)
        kb = 3
        gb = [core.grid(q) for q in rb.problems[:kb]]
        yb, _ = rb.eval(gb)
        ybc = yb.cpu().numpy()
        off, errs_b = 0, []
        for q, g in zip(rb.problems[:kb], gb):
            ref = core.solve_linear(q)["y"]
            errs_b.append(float(np.abs(ybc[off:off + len(g)] - ref).max() / np.abs(ref).max()))
            off += len(g)
        extra["bvp_4096"] = {"ms_per_step": msb, "solves_s": 4096 / (msb / 1000.0),
                             "refine_passes": 2, "rel_err_vs_oracle_max": max(errs_b),
                             "status_ok": bool((rb.status.cpu().numpy() == 0).all())}
        rb.close()
        # single instances at the paper's scale (n = 1e4, m = 50): linear FP64 and
        # mixed, nonlinear y' = 1 - y^2 by Newton (FP64)
        single = {}
        for prec in ("fp64", "mixed"):
            s1 = Batch([ni.cfg2_linear()], precision=prec)
            single["linear_" + prec + "_ms"] = step_ms(s1, s1.run)
            s1.close()
        sn = Batch([ni.cfg2_tanh()], precision="fp64")
        single["tanh_newton_ms"] = step_ms(sn, lambda: sn.newton(max_iter=50, tol=1e-10), reps=2)
        sn.close()
        extra["single_n1e4"] = single
        # long-time single instances at the sizes of Table 12 (n = 5e4, m = 200, FP64;
        # factor, assembly and solve per step): Problem 3 (omega coordinates, 111
        # of 200 eigenpairs kept) and Problem 9 (all 200 kept)
        try:
            extra["long_time_n5e4_m200"] = long_time_breakdown(Batch, ni, torch)
        except Exception as ex:   # a side measurement must not cost the metric line
            extra["long_time_n5e4_m200"] = {"error": repr(ex)[:200]}
        # third- and fourth-order batch (FP64, tabulated coefficients): 1024 instances,
        # n in {1000, 2000}, m in {20, 32}, half of the fourth-order ones with
        # Problem 16's boundary values
        try:
            hp = ni.small_higher(1024, sub=7, n_choices=(1000, 2000), m_choices=(20, 32))
            bh = Batch(hp, precision="fp64")
            msh = step_ms(bh, bh.run)
            _, sth = bh.run()
            torch.cuda.synchronize()
            extra["higher_order_1024"] = {"ms_per_step": msh, "solves_s": len(hp) / (msh / 1000.0),
                                          "status_ok": bool((sth.cpu().numpy() == 0).all())}
            bh.close()
        except Exception as ex:
            extra["higher_order_1024"] = {"error": repr(ex)[:200]}
        # batched Newton family: 64 logistic / Duffing instances, n in [2000, 1e4], FP64
        b5 = Batch(ni.cfg5(), precision="fp64")
        ms5 = step_ms(b5, lambda: b5.newton(max_iter=20, tol=1e-10), reps=2)
        _, st5, it5, _ = b5.newton(max_iter=20, tol=1e-10)
        extra["newton_cfg5"] = {"instances": len(b5.problems), "ms": ms5,
                                "max_iters": int(it5.max().item()),
                                "converged": int((st5 == 0).sum().item())}
        b5.close()
        rate, kk, dt = oracle_rate(probs, args.cpu_seconds)
        cpu_base = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                    "sample": "first %d instances of the workload, numpy FP64 oracle, %.1f s" % (kk, dt)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": workload_config(args, ws),
            "e2e": {"value": ws * B / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "kernel": "k_assemble_tc" if args.precision == "mixed"
                         else "k_assemble_f64", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                         "traffic": (TC_DRAM_BYTES_PER_INSTANCE * B if args.precision == "mixed"
                                     and args.n == 10_000 and args.m == 50 else None),
                         "flops_per_launch": fl, "ms_per_launch": asm_ms},
            "cpu_baseline": cpu_base,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    bt.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def C_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


if __name__ == "__main__":
    main()
