#!/usr/bin/env python
"""Benchmark: PDHG iterations per second of the restarted primal-dual conic solver.

Workload (default): the large mixed-cone LP/SOCP/exp program, n = 1,000,000
variables, m = 500,000 rows, ~10M nonzeros (log-normal row degrees 2-200, N(0,1)
values), 200k nonnegative rows, SOC blocks of dimension 4-64 filling 200k rows,
20k exponential cones, 40k zero rows, known optimum; FP64.  A step is one check
period: 64 PDHG evaluations (primal update, K xhat, dual update + cone
projection, K' yhat) plus one restart / termination check, replayed as one CUDA
graph.  The working set (K, K' and ~15 state vectors, ~0.5 GB) is larger than
the 129 MB L2, so no flush is needed between steps.

One JSON line is printed by rank 0.  Under torchrun each rank runs an
independent replica (the method has no data-path exchange on one instance).
``--impl reference`` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EVALS_PER_STEP = 64
METRIC = "PDHG iters/sec"
WORKLOADS = {
    "mixed_cone_1m": "mixed-cone LP/SOCP/exp, n=1,000,000, m=500,000, ~10M nnz, 200k nonneg rows, "
                     "SOC(4-64) on 200k rows, 20k exp cones, 40k zero rows, known optimum, seed 1",
    "small_socp": "random sparse SOCP, n=2,000, m=1,000, 20k nnz, 500 nonneg rows + 50 SOC(10), seed 0",
    "mixed_cone_literal": "mixed-cone LP/SOCP/exp with the literal cone counts, n=1,000,000, m=2,000,000, ~41M nnz, "
                          "200k nonneg rows, ~50k SOC(4-64) on 1.7M rows, 20k exp cones, 40k zero rows, known "
                          "optimum, seed 1",
    "logistic_exp_200k": "l1 logistic regression as an exp-cone program: 200,000 samples x 2,000 features at "
                         "0.5 % density (N(0,1), labels +-1), 400k exp cones + 200k nonneg rows, n=604,000, "
                         "m=1,400,000, ~5.2M nnz, lam = 0.1 ||X'b||_inf / 2, seed 2",
    "lasso_paper_70k": "Lasso (App. B.2 generator): A 70,000 x 700,000 with 4.9e6 entries U[0,1], lam = "
                       "||A'b||_inf; SOCP n=1,470,002, m=140,003, ~9.9M nnz, one SOC of 70,002 rows, seed 0",
    "fisher_100k": "Fisher market (App. B.1 generator): 100,000 buyers x 1,000 goods, U at 20 % density "
                   "U[0,1]; exp-cone program n=20,200,000, m=401,000, ~40M nnz, 100k exp cones, seed 0",
}


def make_workload(name):
    from paper_2505_00311_gb300 import instances as I
    if name == "mixed_cone_1m":
        return I.mixed_cone(1)
    if name == "small_socp":
        return I.small_socp(0)
    if name == "mixed_cone_literal":
        return I.mixed_cone_literal(1)
    if name == "logistic_exp_200k":
        return I.logistic_exp(2)
    if name == "lasso_paper_70k":
        return I.lasso_paper(0, 70_000, 700_000, 1e-4)
    if name == "fisher_100k":
        return I.fisher_market(0, 100_000, 1000, 0.2)
    raise SystemExit("unknown workload " + name)


def problem_bytes(p):
    bounds = sum(p[k].size * 8 for k in ("lb", "ub") if p.get(k) is not None)
    return (p["row_ptr"].size * 8 + p["col"].size * 4 + p["val"].size * 8 + p["c"].size * 8 + p["h"].size * 8
            + bounds + len(p["cone_types"]) * 16)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline of the dominant kernel
# ---------------------------------------------------------------------------
def algorithmic_bytes(p):
    """Bytes one launch of each kernel class must move at least (FP64 values, int32 indices),
    counting each gathered vector once (it stays in L2)."""
    m, n, nnz = p["m"], p["n"], int(p["row_ptr"][-1])
    types = np.asarray(p["cone_types"])
    dims = np.asarray(p["cone_dims"])
    cone_rows = int(dims[(types == 2) | (types == 3) | (types == 4)].sum())
    return {
        # val + col per nonzero, the binned row pointer and output row index, the gathered
        # input once, the output
        "spmv_K": nnz * 12 + (m + 1) * 4 + m * 4 + n * 8 + m * 8,
        "spmv_KT": nnz * 12 + (n + 1) * 4 + n * 4 + m * 8 + n * 8,
        # reads x, xhat, x0, K'y, K'yhat, K'y0, xsum, c, l, u; writes x, K'y, xsum, xhat
        "primal_update": n * 14 * 8,
        # reads y, yhat, y0, Kx, K xhat (both buffers), Kx0, ysum, h; writes y, Kx, ysum, yhat;
        # plus the row scales of the SOC / exp rows
        "dual_update": m * 13 * 8 + cone_rows * 8,
    }


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2505_00311_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_record(kernel, field="bytes_per_launch"):
    """A per-kernel figure of the committed ncu summary (DRAM bytes per launch, or the
    FP64-pipe activity in % with field="fp64_pipe_active_pct"), if it was taken on this
    source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash():
        return None
    return rec.get(field, {}).get(kernel)


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    return ncu_record(kernel)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def cpu_baseline(p, budget_s=15.0, steps=None):
    import oracle
    o = oracle.Solver(p)
    t0 = time.perf_counter()
    o.run(1)
    one = time.perf_counter() - t0
    n = steps if steps else max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.run(n)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": "%d PDHG evaluations of the FP64 oracle (single thread) after setup and one "
                      "evaluation, same workload" % n, "seconds": dt}


def job_rate(ms, evals, dist=None, device="cpu"):
    """Whole-job rate of independent replicas: every rank ran `evals` evaluations in `ms`
    milliseconds and the job lasts as long as the slowest rank.  Returns (evaluations per
    second over all ranks, the max time in ms)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        world = dist.get_world_size()
    return world * evals / (ms / 1000.0), ms


def bench_config(args, world):
    """The workload description both arms print."""
    return {"workload": WORKLOADS[args.workload], "step": "64 PDHG evaluations + 1 restart check",
            "precision": "fp64", "l2": "working set > L2 (no flush needed)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pdcs", choices=["pdcs", "reference"])
    ap.add_argument("--workload", default="mixed_cone_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run (profiling runs)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-iterate mode measurements")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-programs measurement")
    ap.add_argument("--no-proj", action="store_true", help="skip the standalone projection measurements")
    ap.add_argument("--no-lasso", action="store_true", help="skip the paper-generator Lasso time-to-tolerance runs")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start measurement")
    ap.add_argument("--no-exp", action="store_true",
                    help="skip the exp-cone logistic program (plain vs learned exp root start)")
    ap.add_argument("--batch-count", type=int, default=256, help="Lasso programs in the batched measurement")
    ap.add_argument("--batch-nhi", type=int, default=400, help="largest feature count of the batched Lasso programs")
    ap.add_argument("--batch-seq-sample", type=int, default=0,
                    help="programs of the one-by-one baseline (0: all; fewer: a seeded sample, time scaled up)")
    ap.add_argument("--time-to-tol", default="1e-4,1e-6",
                    help="comma list of tolerances for the time-to-solution runs ('' to skip)")
    ap.add_argument("--ttt-limit", type=float, default=100.0, help="seconds allowed per time-to-tolerance run")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # the FP64 CPU oracle on the same workload: W untimed evaluations, then exactly K
        # timed ones; a step of this arm is one PDHG evaluation (the GPU arm's step of 64
        # evaluations and a check would take ~25 s on one core)
        import oracle
        p = make_workload(args.workload)
        steps = max(1, args.steps)
        o = oracle.Solver(p)
        o.run(args.warmup)
        t0 = time.perf_counter()
        o.run(steps)
        dt = time.perf_counter() - t0
        value = steps / dt
        cb = {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
              "sample": "%d PDHG evaluations of the FP64 oracle (single thread) after setup and %d untimed "
                        "evaluations, same workload" % (steps, args.warmup), "seconds": dt}
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus, "steps": steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * dt / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference", "config": bench_config(args, 1),
                "reference_step": "one PDHG evaluation of the CPU oracle (ms_per_step is per evaluation)",
                "cpu_baseline": cb,
                "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2505_00311_gb300 import build as B
    from paper_2505_00311_gb300 import pdcs as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    p = make_workload(args.workload)
    stream = torch.cuda.Stream()
    solver = P.Solver(p, stream=stream.cuda_stream, spmv_autotune=1)

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (also captures the CUDA graph)
    for _ in range(args.warmup):
        solver.run(EVALS_PER_STEP)
    # per-kernel durations (CUDA events on the solver's stream), one check period
    ktimes, kcounts = solver.kernel_times(EVALS_PER_STEP)
    info0 = solver.info()

    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        solver.run(EVALS_PER_STEP)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    info1 = solver.info()
    launches = info1["kernel_launches"] - info0["kernel_launches"]
    evals = args.steps * EVALS_PER_STEP
    accepted = info1["accepted"] - info0["accepted"]
    # matrix-vector products: K xhat every evaluation, K' yhat after accepted ones, four per check
    matvecs = evals + accepted + 4 * args.steps
    value, ms = job_rate(ms, evals, dist, "cuda")
    rates = {"accepted_iters_per_s": value * accepted / evals, "matvecs_per_s": value * matvecs / evals,
             "accepted_per_step": accepted / args.steps, "matvecs_per_step": matvecs / args.steps,
             "spmv_format": {1: "binned", 2: "sliced"}.get(info1.get("spmv_format"), None)}
    solver.close()

    # end to end through the public API with host buffers: create (H2D + setup),
    # the same number of evaluations, solution read back (D2H)
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = P.Solver(p, stream=stream.cuda_stream, spmv_autotune=1)
        s2.run(evals)
        x, y = s2.solution()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        s2.close()
        e2e = {"value": evals / e2e_s, "unit": "iters/s",
               "h2d_bytes_per_step": int(problem_bytes(p) / args.steps),
               "d2h_bytes_per_step": int((x.size + y.size) * 8 / args.steps),
               "includes": "pdcs_create from host arrays (copy + rescaling + K' build) + pdcs_solve + "
                           "pdcs_get_solution"}

    # time to tolerance: one trajectory per mode, solved to each tolerance in turn (a solve
    # that met a looser tolerance continues towards the next one); wall clock of pdcs_solve,
    # cumulative, setup (pdcs_create) reported apart
    def time_to_tols(**opts):
        tols = sorted((float(t) for t in args.time_to_tol.split(",") if t), reverse=True)
        s3 = P.Solver(p, stream=stream.cuda_stream, time_limit=args.ttt_limit, **opts)
        out, total = [], 0.0
        for tol in tols:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, inf = s3.solve(tol, 4_000_000)
            torch.cuda.synchronize()
            total += time.perf_counter() - t0
            out.append({"tol": tol, "seconds": total, "status": P.STATUS_NAMES.get(st, st),
                        "evaluations": inf["attempts"], "accepted": inf["accepted"], "restarts": inf["restarts"],
                        "fp64_phase": bool(inf["fp64_phase"]), "err": [inf["err_p"], inf["err_d"], inf["err_gap"]],
                        "setup_seconds": inf["setup_seconds"]})
            if st != P.OK:
                break
        s3.close()
        return out

    ttt = time_to_tols(spmv_autotune=1) if args.time_to_tol else []

    # the FP32-iterate mode on the same workload: steady-state rate and time to tolerance
    # (FP32 iterates, FP64 checks, FP64 iterations once the FP32 phase hands over)
    fp32 = None
    if not args.no_fp32:
        s4 = P.Solver(p, stream=stream.cuda_stream, precision=P.PRECISION_FP32, spmv_autotune=1)
        for _ in range(args.warmup):
            s4.run(EVALS_PER_STEP)
        kt32, _ = s4.kernel_times(EVALS_PER_STEP)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            s4.run(EVALS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1)
        phase = s4.info()["fp64_phase"]
        s4.close()
        ttt32 = time_to_tols(precision=P.PRECISION_FP32, spmv_autotune=1) if args.time_to_tol else []
        fp32 = {"value": job_rate(ms32, evals, dist, "cuda")[0], "unit": "iters/s", "ms_per_step": ms32 / args.steps,
                "dtype": "f32 iterates, f64 checks", "still_fp32_phase": phase == 0,
                "kernels_ms_per_launch": kt32, "time_to_tol": ttt32}

    # batched programs: uneven-size Lasso SOCPs solved to 1e-6 in one batch against the
    # plain method solving them one after the other (same instances, same tolerance)
    batch = None
    if not args.no_batch:
        from paper_2505_00311_gb300 import instances as I
        t_gen = time.perf_counter()
        probs = I.lasso_batch(7, args.batch_count, 50, args.batch_nhi)
        t_gen = time.perf_counter() - t_gen
        G = 8
        t_create = time.perf_counter()
        # reflection parameter 1/2 for this family (both arms): with the default 1, 3 of the
        # 256 programs stall with the gap error near 1e-3 for 100k evaluations; all converge at 1/2
        beta_b = 0.5
        solvers = [P.Solver(q, stream=stream.cuda_stream, batch_blocks=G, beta=beta_b) for q in probs]
        t_create = time.perf_counter() - t_create
        bt = P.Batch(solvers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, nconv = bt.solve(1e-6, 100_000)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        bstats = [sv.info() for sv in solvers]
        evals_b = max(b["attempts"] for b in bstats)
        bt.close()
        for sv in solvers:
            sv.close()
        nonconv = [{"program": k, "n": int(probs[k]["n"]), "evaluations": bstats[k]["attempts"],
                    "err": [bstats[k]["err_p"], bstats[k]["err_d"], bstats[k]["err_gap"]]}
                   for k in range(len(probs)) if bstats[k]["status"] != P.OK][:10]
        seq_idx = list(range(len(probs)))
        if 0 < args.batch_seq_sample < len(probs):
            seq_idx = sorted(np.random.default_rng(17).choice(len(probs), args.batch_seq_sample, replace=False).tolist())
        t_seq, nseq, evals_s = 0.0, 0, 0
        for q in (probs[k] for k in seq_idx):
            sv = P.Solver(q, stream=stream.cuda_stream, beta=beta_b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st1, inf1 = sv.solve(1e-6, 100_000)
            torch.cuda.synchronize()
            t_seq += time.perf_counter() - t0
            nseq += st1 == P.OK
            evals_s += inf1["attempts"]
            sv.close()
        scale = len(probs) / len(seq_idx)
        batch = {"workload": "%d Lasso SOCPs (App. B.2 form), n ~ U{50..%d} features, m = n/2, dense N(0,1) "
                             "design, tol 1e-6, FP64" % (len(probs), args.batch_nhi),
                 "nnz_total": int(sum(int(q["row_ptr"][-1]) for q in probs)),
                 "beta": beta_b, "generate_seconds": t_gen, "create_seconds": t_create,
                 "batched_seconds": t_batch, "batched_converged": nconv, "batched_lockstep_evaluations": evals_b,
                 "not_converged": nonconv,
                 "sequential_programs": len(seq_idx), "sequential_seconds": t_seq * scale,
                 "sequential_seconds_measured": t_seq, "sequential_converged": nseq,
                 "sequential_total_evaluations": evals_s,
                 "speedup": t_seq * scale / t_batch if t_batch > 0 else None}

    # standalone cone projections (Sec. 4's strategy comparison, Fig. 3 stand-in): 2e8 entries
    # as SOC blocks of several sizes, and 2e6 exp cones, unscaled (D = I) and with scales
    # exp(N(0, 0.5^2)); a projection plan per layout (built before the timed runs), whose runs
    # only enqueue kernels; bytes: read v (and d) and write the result once
    proj = None
    if not args.no_proj:
        proj = []
        g = torch.Generator(device="cuda").manual_seed(3)
        total = 200_000_000
        peak = measured_peaks().get("hbm_gbs")

        def timed(fn, reps=5):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        v = torch.randn(total, device="cuda", dtype=torch.float64, generator=g)
        dsc = torch.exp(0.5 * torch.randn(total, device="cuda", dtype=torch.float64, generator=g))
        out = torch.empty_like(v)
        for nblk in [10, 1_000, 100_000, 10_000_000]:
            dim = total // nblk
            types = np.full(nblk, P.CONE_SOC, np.int32)
            dims = np.full(nblk, dim, np.int64)
            plan = P.ProjPlan(nblk * dim, types, dims, stream.cuda_stream)
            for scaled in (False, True):
                dp = dsc.data_ptr() if scaled else 0
                pms = timed(lambda: plan.run(v.data_ptr(), dp, 0, out.data_ptr(), stream.cuda_stream))
                byt = nblk * dim * (24 if scaled else 16)
                proj.append({"cones": "SOC", "count": nblk, "dim": dim, "scaled": scaled, "ms": pms,
                             "GBps": byt / (pms * 1e-3) / 1e9, "frac_of_hbm": byt / (pms * 1e-3) / 1e9 / peak
                             if peak else None})
            if plan.check(stream.cuda_stream) != P.OK:
                raise SystemExit("projection plan: a team wait gave up")
            plan.close()
        ne = 2_000_000
        types = np.full(ne, P.CONE_EXP, np.int32)
        dims = np.full(ne, 3, np.int64)
        plan = P.ProjPlan(3 * ne, types, dims, stream.cuda_stream)
        for scaled in (False, True):
            dp = dsc.data_ptr() if scaled else 0
            pms = timed(lambda: plan.run(v.data_ptr(), dp, 0, out.data_ptr(), stream.cuda_stream))
            byt = 3 * ne * (24 if scaled else 16)
            proj.append({"cones": "EXP", "count": ne, "dim": 3, "scaled": scaled, "ms": pms,
                         "cones_per_s": ne / (pms * 1e-3), "GBps": byt / (pms * 1e-3) / 1e9})
        plan.close()
        del v, dsc, out

    # learned warm start on a parametric portfolio family (400 assets, 10 factors): a network
    # trained on 160 batched solves predicts (log omega, y) from a summary of the returns; 24
    # held-out instances solved to 1e-6 cold and warm, one at a time (wall clock of pdcs_solve,
    # prediction time included in the warm arm), with FP32 and BF16 tensor-core predictions
    warm = None
    if not args.no_warm:
        from paper_2505_00311_gb300 import instances as I
        fam = I.portfolio_family(0, 400, 10)
        sizes = [17, 256, 256, 23]

        def solve_batch(seeds):
            svs = [P.Solver(I.portfolio_socp(fam, I.portfolio_mu(fam, sd)), stream=stream.cuda_stream, batch_blocks=4)
                   for sd in seeds]
            bt = P.Batch(svs)
            bt.solve(1e-6, 200_000)
            out = [(sv.solution(), sv.info()) for sv in svs]
            bt.close()
            for sv in svs:
                sv.close()
            return out

        train = list(range(160))
        t0 = time.perf_counter()
        res = solve_batch(train)
        t_data = time.perf_counter() - t0
        Xtr = np.stack([I.portfolio_features(fam, I.portfolio_mu(fam, sd)) for sd in train])
        Ytr = np.stack([np.concatenate([[np.log(inf["omega"])], y]) for (x, y), inf in res])
        mu_x, sd_x = Xtr.mean(axis=0), Xtr.std(axis=0) + 1e-12
        mu_y, sd_y = Ytr.mean(axis=0), Ytr.std(axis=0) + 1e-12
        t0 = time.perf_counter()
        Wn, _ = P.mlp_train(sizes, (Xtr - mu_x) / sd_x, (Ytr - mu_y) / sd_y, P.mlp_init(sizes, 0), steps=3000,
                            batch=64, lr=1e-3, seed=7)
        t_train = time.perf_counter() - t0
        held = list(range(1000, 1024))
        arms = {}
        for arm in ("cold", "warm_fp32", "warm_bf16"):
            w_secs, w_evals, w_conv = 0.0, 0, 0
            for sd in held:
                q = I.portfolio_socp(fam, I.portfolio_mu(fam, sd))
                sv = P.Solver(q, stream=stream.cuda_stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if arm != "cold":
                    f = ((I.portfolio_features(fam, I.portfolio_mu(fam, sd)) - mu_x) / sd_x)[None, :]
                    fwd = P.mlp_forward if arm == "warm_fp32" else P.mlp_forward_bf16
                    pr = fwd(sizes, f, Wn)[0] * sd_y + mu_y
                    sv.warm_start(None, pr[1:].astype(np.float64), float(np.exp(pr[0])))
                st1, inf1 = sv.solve(1e-6, 200_000)
                torch.cuda.synchronize()
                w_secs += time.perf_counter() - t0
                w_evals += inf1["attempts"]
                w_conv += st1 == P.OK
                sv.close()
            arms[arm] = {"seconds": w_secs, "evaluations": w_evals, "converged": w_conv}
        warm = {"workload": "portfolio SOCP family, 400 assets, 10 factors (budget, box, ||F'x|| <= gamma), "
                            "24 held-out instances to 1e-6 one at a time; network 17-256-256-23 trained on 160 "
                            "batched solves", "training_solves_seconds": t_data, "training_seconds": t_train,
                **arms}

    # the paper's Lasso workload (Sec. 5.3, App. B.2) at 7e4 x 7e5 (4.9e6 entries of A, one SOC
    # of 70,002 rows projected grid-wise): time to 1e-3 and 1e-6 (the paper's two accuracy
    # levels), FP64, wall clock of pdcs_solve, setup apart
    lasso = None
    if not args.no_lasso:
        from paper_2505_00311_gb300 import instances as I
        q = I.lasso_paper(0, 70_000, 700_000, 1e-4)
        sl = P.Solver(q, stream=stream.cuda_stream, time_limit=args.ttt_limit)
        ktl, _ = sl.kernel_times(EVALS_PER_STEP)
        sl.close()
        sl = P.Solver(q, stream=stream.cuda_stream, time_limit=args.ttt_limit)
        inf = sl.info()
        lasso = {"workload": "Lasso (App. B.2 generator), A 70,000 x 700,000, 4.9e6 entries U[0,1], "
                             "lam = ||A'b||_inf; SOCP n = %d, m = %d, nnz = %d, one SOC of %d rows" %
                             (q["n"], q["m"], int(q["row_ptr"][-1]), int(q["cone_dims"][-1])),
                 "soc_grid_cones": inf["soc_grid_cones"], "setup_seconds": inf["setup_seconds"],
                 "kernels_ms_per_launch": ktl, "time_to_tol": []}
        total_s = 0.0
        for tol in (1e-3, 1e-6):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, inf = sl.solve(tol, 10_000_000)
            torch.cuda.synchronize()
            total_s += time.perf_counter() - t0
            lasso["time_to_tol"].append({"tol": tol, "seconds": total_s, "status": P.STATUS_NAMES.get(st, st),
                                         "evaluations": inf["attempts"],
                                         "err": [inf["err_p"], inf["err_d"], inf["err_gap"]]})
            if st != P.OK:
                break
        sl.close()
        # the same Lasso in the appendix's own form: (w, r, y) in K_rsoc as a primal cone block,
        # the m + 1 zero rows only (each solve call limited to half the time-to-tolerance limit)
        qk = I.lasso_paper_kp(0, 70_000, 700_000, 1e-4)
        sk = P.Solver(qk, stream=stream.cuda_stream, time_limit=args.ttt_limit / 2)
        kp = {"form": "primal cone block of %d variables, %d rows, nnz = %d" %
                      (int(qk["pcone_dims"][0]), qk["m"], int(qk["row_ptr"][-1])),
              "setup_seconds": sk.info()["setup_seconds"], "time_to_tol": []}
        total_s = 0.0
        for tol in (1e-3, 1e-6):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, inf = sk.solve(tol, 10_000_000)
            torch.cuda.synchronize()
            total_s += time.perf_counter() - t0
            kp["time_to_tol"].append({"tol": tol, "seconds": total_s, "status": P.STATUS_NAMES.get(st, st),
                                      "evaluations": inf["attempts"],
                                      "err": [inf["err_p"], inf["err_d"], inf["err_gap"]]})
            if st != P.OK:
                break
        sk.close()
        lasso["primal_cone_form"] = kp

    # the exp-cone-heavy program (l1 logistic regression, 400k exp cones), plain exp root
    # search against the learned starting point: the first evaluation (no cached roots), the
    # steady-state rate and the time to 1e-6
    exp_heavy = None
    if not args.no_exp:
        from paper_2505_00311_gb300 import instances as I
        q = I.logistic_exp(2)
        rng = np.random.default_rng(11)
        v = rng.normal(size=(1_000_000, 3))
        d = np.exp(rng.normal(0.0, 0.5, (1_000_000, 3)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        feats, target = P.exp_mlp_dataset(v, d)
        w_mlp, _ = P.exp_mlp_train(feats, target, P.exp_mlp_init(0), steps=4000, batch=4096, lr=2e-3, seed=5)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        exp_heavy = {"workload": WORKLOADS["logistic_exp_200k"],
                     "network": {"pairs": int(target.size), "steps": 4000, "batch": 4096, "seconds": train_s,
                                 "data": "case-4 roots of the plain search for 1M N(0,1) 3-vectors with scales "
                                         "exp(N(0, 0.5^2))"}}
        for name, w in (("plain", None), ("learned", w_mlp)):
            s6 = P.Solver(q, stream=stream.cuda_stream, spmv_autotune=1, exp_mlp=w)
            first, _ = s6.kernel_times(1)
            for _ in range(args.warmup):
                s6.run(EVALS_PER_STEP)
            kt6, _ = s6.kernel_times(EVALS_PER_STEP)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                s6.run(EVALS_PER_STEP)
            e1.record(stream)
            torch.cuda.synchronize()
            ms6 = e0.elapsed_time(e1)
            s6.close()
            s7 = P.Solver(q, stream=stream.cuda_stream, time_limit=args.ttt_limit, spmv_autotune=1, exp_mlp=w)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, inf = s7.solve(1e-6, 2_000_000)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            s7.close()
            exp_heavy[name] = {
                "first_evaluation_dual_update_ms": first["dual_update"],
                "value": job_rate(ms6, evals, dist, "cuda")[0], "unit": "iters/s", "ms_per_step": ms6 / args.steps,
                "dual_update_ms": kt6["dual_update"], "kernels_ms_per_launch": kt6,
                "time_to_1e-6": {"seconds": dt, "status": P.STATUS_NAMES.get(st, st), "evaluations": inf["attempts"],
                                 "restarts": inf["restarts"], "err": [inf["err_p"], inf["err_d"], inf["err_gap"]],
                                 "setup_seconds": inf["setup_seconds"]}}

    if rank != 0:
        return
    # roofline of the dominant kernel.  On this GPU the FP64 pipe (2 thread operations per
    # cycle per SM) binds every kernel of the path before HBM does: even the vector updates
    # do ~15 FP64 operations per 112 bytes.  The FP64 work of a launch is the FP64 floating-
    # point operations its algorithm executes (FMA = 2), counted by ncu on this source
    # (profiles/ncu_traffic.json); without that record the HBM view is the fallback.
    alg = algorithmic_bytes(p)
    if info0.get("fuse_primal"):  # the K' product carries the primal update; primal_update only runs
        alg["spmv_KT"] += alg["primal_update"]  # after rejected steps and checks
        alg["primal_update"] = 0
    per_step_ms = {k: ktimes[k] * kcounts[k] / 1.0 for k in alg}
    dom = max(alg, key=lambda k: per_step_ms[k])
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    fp64_peak = 2 * 2 * sms * mhz * 1e6 / 1e12  # TFLOP/s: 2 FP64 ops/cycle/SM, FMA = 2 FLOP
    kern = {}
    for k in ktimes:
        rec = {"ms_per_launch": ktimes[k], "launches_per_step": kcounts[k]}
        if k in alg and ktimes[k] > 0 and alg[k] > 0:
            rec["GBps"] = alg[k] / (ktimes[k] * 1e-3) / 1e9
            rec["frac_of_hbm"] = rec["GBps"] / hbm if hbm else None
            fl = ncu_record(k, "fp64_flops_per_launch")
            if fl:
                rec["fp64_TFLOPs"] = fl / (ktimes[k] * 1e-3) / 1e12
                rec["frac_of_fp64"] = rec["fp64_TFLOPs"] / fp64_peak
        kern[k] = rec
    hbm_view = {"achieved": kern[dom].get("GBps"), "peak": hbm, "unit": "GB/s", "frac": kern[dom].get("frac_of_hbm"),
                "algorithmic_bytes_per_launch": alg[dom]}
    flops = ncu_record(dom, "fp64_flops_per_launch")
    if flops:
        roof = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["fp64_TFLOPs"], "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": kern[dom]["frac_of_fp64"], "traffic": ncu_traffic(dom),
                "peak_source": "derived: 2 FP64 thread operations per cycle per SM (ncu peak_sustained) x %d SMs x "
                               "%.0f MHz, FMA = 2 FLOP" % (sms, mhz),
                "flops_per_launch": flops, "flops_source": "FP64 operations executed per launch (ncu, this source)",
                "ms_per_launch": ktimes[dom], "hbm_view": hbm_view, "kernels": kern}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": hbm_view["achieved"], "peak": hbm, "unit": "GB/s",
                "frac": hbm_view["frac"], "traffic": ncu_traffic(dom),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "unavailable",
                "algorithmic_bytes_per_launch": alg[dom], "ms_per_launch": ktimes[dom], "kernels": kern}
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(p)
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": bench_config(args, world),
            "rates": rates, "clocks": clk, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
            "time_to_tol": ttt, "fp32_iterates": fp32, "batched_programs": batch, "projections": proj, "paper_lasso": lasso, "warm_start": warm,
            "exp_heavy": exp_heavy}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
