#!/usr/bin/env python
"""Throughput of the GenCD hot path on GB300: non-zeros processed per second.

One step = one Thread-Greedy GenCD iteration (Algorithm 1, Table 2) over the
whole synthetic workload: Select (all columns), Propose (streaming pass over
X computing g, the Eq. 7 step and the Eq. 9 proxy for every column), the
convergence quantities of the start state (KKT violation and objective),
Accept (best proxy per partition), Update (atomic scatter into z) and the
refresh of u on the touched rows.

Workload: logistic l1 problem with n=1,000,000 rows, k=4,000,000 columns,
Zipf(1.1) column lengths capped at 50,000 (2.0e8 non-zeros), log-normal values
with unit-norm columns, 2,000 planted weights, lambda = 0.05 lambda_max.

  value   nnz processed per second with X resident in HBM (CUDA events on the
          library's stream, max over ranks)
  e2e     the same metric through the C ABI from pinned host buffers: each step
          creates the problem from host memory (H2D of X and y), runs one
          iteration and reads the objective and KKT value back (D2H)

  serving  p50/p99 latency and solves/s of a config-5 request stream served
          with concurrent requests and one at a time (run_serve)
  regularisation_path  batched solves/s of a cross-validated lambda path on
          config 4 (5 row folds x 32 lambdas, one gencd_batch over X) beside
          the same 160 solves through gencd_solve one at a time (run_path)

`--impl reference` times the FP64 CPU oracle on the host cores instead (the
paper's method has no other runnable implementation).  Under torchrun every
rank runs an independent replica (the path is replicated, not sharded).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD_DESC = ("logistic l1, n=1,000,000, k=4,000,000, Zipf(1.1) column nnz capped at 50,000, "
                 "2.0e8 nnz, log-normal unit-norm columns, lambda=0.05*lambda_max, seed 0")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gencd", choices=["gencd", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16", "binary"],
                    help="storage mode of X (bf16 and binary compute in FP32; binary runs on the "
                         "workload's pattern with 1/sqrt(nnz_j) values)")
    ap.add_argument("--variant", default="thread_greedy", choices=["thread_greedy", "greedy"])
    ap.add_argument("--blocks", type=int, default=1024)
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the full workload (tests)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--propose-split", type=int, default=-1,
                    help="streaming propose schedule (-1: the autotuner's; 0: two kernels; 20-31: fused split), "
                         "e.g. to profile one form under ncu, whose replays distort the autotuner's timings")
    ap.add_argument("--legs", type=int, default=1,
                    help="also time config 2 in the other storage modes and variants, and config 1 (0/1)")
    ap.add_argument("--leg-steps", type=int, default=30, help="timed iterations of each config-2 leg")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="time limit of the FP64 reference solve that gives P* for the time-to-1e-6 run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--target-check", type=int, default=10,
                    help="iterations between objective checks of the time-to-1e-6 run (0: skip it)")
    ap.add_argument("--target-max-iter", type=int, default=5000)
    # regularisation path (batched solves over one X against one solve per call)
    ap.add_argument("--path", type=int, default=1, help="add the regularisation-path measurement (0/1)")
    ap.add_argument("--path-loss", default="squared", choices=["squared", "logistic"])
    ap.add_argument("--path-scale", type=float, default=0.1, help="fraction of config 4's size")
    ap.add_argument("--path-ratio-long", type=float, default=1e-3,
                    help="smallest lambda / lambda_max of the second, batched-only run (0: skip it)")
    ap.add_argument("--path-max-iter-long", type=int, default=100_000)
    ap.add_argument("--path-slots", type=int, default=32)
    ap.add_argument("--path-blocks", type=int, default=1024)
    ap.add_argument("--path-check", type=int, default=5)
    ap.add_argument("--path-tol-rel", type=float, default=1e-3, help="KKT <= tol_rel lambda (when --path-tol-gap is 0)")
    ap.add_argument("--path-tol-gap", type=float, default=8e-7,
                    help="stop each solve at this relative duality gap (FP32 sums: certified to ~1e-6 in FP64)")
    ap.add_argument("--path-handoff", type=float, default=0.5,
                    help="a fold's next solve starts once KKT <= handoff * lambda (0: after convergence)")
    ap.add_argument("--path-max-iter", type=int, default=100_000)
    ap.add_argument("--path-ratio", type=float, default=1e-2,
                    help="smallest lambda / lambda_max of the path (below ~1/250 on this workload the solutions "
                         "near interpolation and Thread-Greedy stalls)")
    ap.add_argument("--path-plain", type=int, default=5,
                    help="also time the one-solve-per-call form on this many folds' chains (0: skip it)")
    ap.add_argument("--serve", type=int, default=1, help="add the serving-stream measurement (0/1)")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-workers", type=int, default=8, help="slots: requests in flight at most")
    ap.add_argument("--serve-tol", type=float, default=1e-3,
                    help="per-request KKT tolerance relative to lambda (when --serve-tol-gap is 0)")
    ap.add_argument("--serve-tol-gap", type=float, default=8e-7, help="per-request relative duality gap")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="arrival rate of the sustained run, as a fraction of the saturated run's solves/s")
    ap.add_argument("--batch-step", type=int, default=0, metavar="SLOTS",
                    help="time only the batched step on config 4 with SLOTS active slots (profiling entry point)")
    return ap.parse_args()


def load_problem(scale, precision="f32"):
    prob = workloads.config2("logistic") if scale >= 1.0 else workloads.config2_scaled(scale, "logistic")
    return workloads.binarized(prob) if precision == "binary" else prob


# bytes of one stored value of X per storage mode
VALUE_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "binary": 0}


def stored_values_host(val, precision):
    """The values of X as the storage mode holds them, as float64 (numpy /
    PyTorch CPU conversions: FP32 round to nearest even, then bfloat16 round
    to nearest even).  Used to give the FP64 reference solve the same X as the
    timed run."""
    if precision == "f64":
        return np.asarray(val, np.float64)
    v32 = np.asarray(val, np.float32)
    if precision == "bf16":
        import torch

        return torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    return v32.astype(np.float64)


def host_info():
    """Host cores and CPU model of the machine the CPU baseline runs on."""
    info = {"nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
            else os.cpu_count(), "machine": os.uname().machine, "cpu_model": None}
    try:
        import subprocess

        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = {line.split(":", 1)[0].strip(): line.split(":", 1)[1].strip()
                  for line in out.splitlines() if ":" in line}
        info["cpu_model"] = fields.get("Model name") or fields.get("Vendor ID")
        if fields.get("Vendor ID") and fields.get("Model name"):
            info["cpu_model"] = fields["Vendor ID"] + " " + fields["Model name"]
    except (OSError, ValueError):
        pass
    if info["cpu_model"] is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    info["cpu_model"] = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return info


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic(kernel_srcs, precision):
    """DRAM bytes per launch of the streaming propose from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    h = hashlib.sha256()
    for src in kernel_srcs:
        h.update(open(src, "rb").read())
    src_hash = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"propose_all_config2_{precision}.md")
    try:
        text = open(path).read()
    except OSError:
        return None, src_hash
    fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("source_sha256", "dram_bytes_per_launch")))
    if fields.get("source_sha256", "").strip() != src_hash:
        return None, src_hash
    try:
        return float(fields["dram_bytes_per_launch"].strip()), src_hash
    except (KeyError, ValueError):
        return None, src_hash


class ClockSampler:
    """Samples the SM clock and the clock-event (throttle) reasons of one GPU
    every ~2 ms during the timed region, through NVML (read-only queries)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes

        self.C = ctypes
        self.samples = []
        self.max_mhz = None
        self.stop_flag = threading.Event()
        self.thread = None
        self.nvml = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                return
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.nvml, self.h = nv, h
        except (OSError, AttributeError):
            self.nvml = None

    def _loop(self):
        C = self.C
        clk, rs = C.c_uint(), C.c_ulonglong()
        while not self.stop_flag.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, C.byref(clk)) == 0 and \
                    self.reason_fn(self.h, C.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(0.002)

    def start(self):
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()

    def stop(self):
        self.stop_flag.set()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [c for c, _ in self.samples]
        reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(sm), "source": "nvml" if self.nvml else "unavailable"}


def reduce_over_ranks(max_vals, sum_vals, device):
    """Max over ranks of max_vals and sum of sum_vals (identity on one rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in max_vals], [float(v) for v in sum_vals]
    mx = torch.tensor([float(v) for v in max_vals], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in sum_vals], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_omp_rate(sp, lam, blocks, iters, threads, orc=None):
    """Thread-Greedy iterations (B partitions) of the OpenMP baseline
    (Section 4.2's design, FP64) from w = 0 on the full stored workload `sp`
    with `threads` threads; returns (nnz/s, seconds, iterations)."""
    import oracle

    orc = orc or oracle.Oracle(sp, lam)
    s = oracle.OmpSolver(orc, threads=threads)
    t0 = time.perf_counter()
    _, nnz, it = s.iterate(iters, B=blocks)
    el = time.perf_counter() - t0
    s.close()
    return nnz / el, el, it


def cpu_baseline_leg(sp, lam, blocks, w_ref):
    """The CPU baseline (rank 0, one GPU): the OpenMP baseline timed on the
    host's cores, at 1 thread and at all of them, on the whole workload; and
    the oracle's FP64 certificate (KKT violation, duality gap) of the
    reference point the time-to-1e-6 run measured against."""
    import oracle

    info = host_info()
    orc = oracle.Oracle(sp, lam)
    out = {"kind": "oracle", "impl": "OpenMP Thread-Greedy (Section 4.2: static schedule, atomic z), FP64",
           "unit": "nnz/s", "same_config": True, **info}
    try:
        threads = oracle.omp_lib().omp_solver_max_threads()
        r1, el1, it1 = cpu_omp_rate(sp, lam, blocks, 2, 1, orc)
        rT, elT, itT = cpu_omp_rate(sp, lam, blocks, 6, threads, orc)
        out.update({"value": rT, "cores": int(threads), "value_1_thread": r1,
                    "sample": f"{itT} Thread-Greedy iterations (B={blocks}) of the whole workload from w = 0 "
                              f"on {threads} threads in {elT:.1f} s; {it1} on 1 thread in {el1:.1f} s"})
    except Exception as e:  # noqa: BLE001 -- e.g. no OpenMP on the host
        out.update({"value": None, "cores": None, "unavailable": f"{type(e).__name__}: {e}"})
    cert = None
    if w_ref is not None:
        t0 = time.perf_counter()
        z = orc.fitted(w_ref)
        P = orc.objective(w_ref, z)
        kkt = orc.kkt(w_ref, z)
        gap = orc.duality_gap(w_ref, z)
        cert = {"objective": P, "kkt": kkt, "kkt_over_lambda": kkt / lam, "duality_gap": gap,
                "rel_gap": gap / P, "seconds": time.perf_counter() - t0}
    return out, cert


PATH_FOLDS, PATH_LAMBDAS = 5, 32


def _certify_path(gb, prob, fold, F, lam, W, stream):
    """Relative duality gaps (FP64 arithmetic on the device: an FP64 problem
    per training set on the FP32-stored values, set to each solve's w) of the
    F x L solves W[f, t]: each bounds (P(w) - P*) / P(w) of that solve."""
    out = np.full(lam.shape, np.nan)
    for f in range(F):
        sub = workloads.row_subset(prob, np.flatnonzero(fold != f))
        val = sub.val.astype(np.float32).astype(np.float64)  # the batch stores X in FP32
        with gb.Problem(n=sub.n, k=sub.k, col_ptr=sub.col_ptr, row_idx=sub.row_idx, val=val, y=sub.y,
                        loss=sub.loss, precision="f64", stream=stream.cuda_stream) as q:
            for t in range(lam.shape[1]):
                q.set_lambda(lam[f, t])
                q.set_w(W[f, t])
                gap, primal, _ = q.duality_gap()
                out[f, t] = gap / abs(primal) if primal != 0 else gap
    return out


def run_path(args, gb, stream):
    """A cross-validated regularisation path on config 4 (--path-scale of its
    size): 5 row folds x 32 lambdas, each fold's lambda_max down to
    --path-ratio lambda_max, every solve to a relative duality gap of
    --path-tol-gap (or to KKT <= --path-tol-rel lambda), warm started along
    each fold's path.  Batched: one gencd_batch over X runs
    all 160 solves (X streamed once per step for every live solve).  Plain:
    one FP32 problem per fold, one gencd_solve per lambda, warm started by the
    problem's own w.  Both forms' solutions are certified in FP64 on the
    device (relative duality gap of every solve: equal accuracy is checked,
    not assumed).  A second batched run goes to --path-ratio-long
    lambda_max."""
    import torch

    prob = workloads.config4(args.path_loss, seed=0, scale=args.path_scale)
    F, L = PATH_FOLDS, PATH_LAMBDAS
    fold = workloads.cv_folds(prob.n, F, seed=0)

    def batched(ratio, max_iter):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = gb.Batch(prob, fold=fold, nfolds=F, slots=args.path_slots, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        lam = np.stack([workloads.lambda_grid(b.lambda_max(f), L, ratio) for f in range(F)])
        b.set_params(variant="thread_greedy", blocks=args.path_blocks, check_every=args.path_check,
                     max_iter=max_iter, tol_kkt=0.0, tol_gap=args.path_tol_gap)
        tol_rel = 0.0 if args.path_tol_gap > 0 else args.path_tol_rel
        b.path(list(range(F)), lam[:, :1], tol_rel=tol_rel)  # warm-up: capture, autotuning, lambda_max
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs, W, tot = b.path(list(range(F)), lam, handoff=args.path_handoff, warm=True, want_w=True,
                              tol_rel=tol_rel)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        sched = b.schedule()
        b.close()
        st_b = np.array([r["status"] for r in recs])
        res = {"seconds": el, "solves_per_s": F * L / el, "create_s": t_create, "slots": args.path_slots,
               "blocks": args.path_blocks, "handoff": args.path_handoff, "steps": int(tot.iters),
               "updates": int(tot.updates), "nnz_processed": int(tot.nnz_processed),
               "converged": int((st_b == 0).sum()), "converged_by_lambda": (st_b.reshape(F, L) == 0).sum(0).tolist(),
               "iters_per_solve": float(np.mean([r["iters"] for r in recs])),
               "max_group": int(max(r["group"] for r in recs)),
               "schedule": {"spmm_kind": sched[0], "update_kind": sched[1], "candidates_ms": sched[2]}}
        return res, lam, np.array([r["objective"] for r in recs]).reshape(F, L), st_b.reshape(F, L), W

    stop = (f"relative duality gap <= {args.path_tol_gap:g} per solve" if args.path_tol_gap > 0 else
            f"KKT <= {args.path_tol_rel:g} lambda per solve")
    out = {"workload": f"config 4 ({prob.name}), {F} row folds x {L} lambdas (lambda_max -> "
                       f"{args.path_ratio:g} lambda_max), {args.path_loss} loss, {stop}, warm starts",
           "solves": F * L, "stop": stop}
    res_b, lam, P_b, st_b, W_b = batched(args.path_ratio, args.path_max_iter)
    out["batched"] = res_b
    gaps_b = _certify_path(gb, prob, fold, F, lam, W_b.reshape(F, L, -1), stream)
    out["batched"]["certified_rel_gap_max"] = float(np.nanmax(gaps_b[st_b == 0])) if (st_b == 0).any() else None
    if args.path_plain:
        # the plain form on the first --path-plain folds' chains (default: all
        # of them, the batched form's work; the folds' chains differ in
        # difficulty, so a subset would not compare like with like)
        Fp = max(1, min(F, args.path_plain))
        subs = [workloads.row_subset(prob, np.flatnonzero(fold != f)) for f in range(Fp)]  # host prep, untimed
        P_p = np.zeros((Fp, L))
        st_p = np.zeros((Fp, L), np.int64)
        it_p = np.zeros((Fp, L), np.int64)
        W_p = np.zeros((Fp, L, prob.k))
        t_plain = t_pcreate = 0.0
        for f in range(Fp):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p = gb.Problem(subs[f], precision="f32", stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t_pcreate += time.perf_counter() - t0
            t0 = time.perf_counter()
            for t in range(L):
                p.set_lambda(lam[f, t])
                gap_mode = args.path_tol_gap > 0
                p.set_params(variant="thread_greedy", blocks=args.path_blocks,
                             tol_kkt=0.0 if gap_mode else args.path_tol_rel * lam[f, t], tol_gap=args.path_tol_gap,
                             check_every=2 * args.path_check if gap_mode else args.path_check,
                             max_iter=args.path_max_iter)
                r = p.solve()
                P_p[f, t], st_p[f, t], it_p[f, t] = r.objective, r.status, r.iters
                W_p[f, t] = p.w()  # copy out (host), outside nothing: included in the plain form's time
            torch.cuda.synchronize()
            t_plain += time.perf_counter() - t0
            p.close()
        ok = (st_p == 0) & (st_b[:Fp] == 0)
        gaps_p = _certify_path(gb, prob, fold, Fp, lam[:Fp], W_p, stream)
        out["plain"] = {"seconds": t_plain, "solves": Fp * L, "solves_per_s": Fp * L / t_plain,
                        "create_s": t_pcreate, "converged": int((st_p == 0).sum()),
                        "iters_per_solve": float(it_p.mean()),
                        "certified_rel_gap_max": float(np.nanmax(gaps_p[st_p == 0])) if (st_p == 0).any() else None,
                        "folds": Fp}
        out["speedup"] = res_b["solves_per_s"] / out["plain"]["solves_per_s"]
        out["speedup_with_create"] = (F * L / (res_b["seconds"] + res_b["create_s"])) / \
            (Fp * L / (t_plain + t_pcreate))
        rel = np.abs(P_b[:Fp] - P_p) / np.abs(P_p)
        out["max_rel_objective_diff"] = float(rel[ok].max()) if ok.any() else None
    if args.path_ratio_long > 0:
        res_l, lam_l, _, st_l, W_l = batched(args.path_ratio_long, args.path_max_iter_long)
        gaps_l = _certify_path(gb, prob, fold, F, lam_l, W_l.reshape(F, L, -1), stream)
        res_l["certified_rel_gap_max"] = float(np.nanmax(gaps_l[st_l == 0])) if (st_l == 0).any() else None
        res_l["lambda_ratio"] = args.path_ratio_long
        out["batched_to_lambda_max_over_1000"] = res_l
    return out


def run_serve(args, gb):
    """Config 5: independent requests (n in [1e3, 2e5], k in [1e3, 1e6]
    log-uniform, 5-100 nnz per column, squared or logistic loss, lambda =
    U[0.01, 0.3] lambda_max), FP32, each solved by Thread-Greedy to KKT <=
    --serve-tol lambda.  Served (a) arriving as a Poisson process at 200/s
    with --serve-workers slots (the queue grows: the served rate is the
    capacity), (b) arriving at --serve-load of that capacity (latency at a
    sustainable rate) and (c) at 200/s with one slot (one solve at a time)."""
    problems, fracs, arrivals = workloads.serving_stream(args.serve_requests, rate=200.0, seed=0)
    params = dict(variant="thread_greedy", blocks=1024, max_iter=100_000, check_every=10, tol_kkt=0.0,
                  tol_gap=args.serve_tol_gap)

    def summary(res, rate):
        lat = np.array([r["end"] - r["arrival"] for r in res])
        wait = np.array([r["start"] - r["arrival"] for r in res])
        span = max(r["end"] for r in res) - min(r["arrival"] for r in res)
        return {"arrival_rate": rate, "solves_per_s": len(res) / span, "p50_ms": 1000.0 * float(np.percentile(lat, 50)),
                "p99_ms": 1000.0 * float(np.percentile(lat, 99)), "seconds": span,
                "queue_wait_p50_ms": 1000.0 * float(np.percentile(wait, 50)),
                "queue_wait_max_ms": 1000.0 * float(wait.max()),
                "converged": int(sum(r["status"] == 0 for r in res)), "requests": len(res)}

    tol_rel = 0.0 if args.serve_tol_gap > 0 else args.serve_tol
    if tol_rel > 0:
        params["tol_gap"] = 0.0

    def serve(arr, workers):
        return gb.gencd_serve(problems, fracs, arr, workers=workers, hbm_fraction=0.5, tol_rel=tol_rel,
                              **params)[0]

    gb.gencd_serve(problems[:2], fracs[:2], arrivals[:2] * 0, workers=2, tol_rel=tol_rel, **params)  # warm-up
    mix = serve(arrivals, args.serve_workers)
    sat = summary(mix, 200.0)
    rate = max(1e-3, args.serve_load * sat["solves_per_s"])  # a rate the slots sustain
    gaps = np.random.Generator(np.random.PCG64(1)).exponential(1.0 / rate, len(problems))
    arr_load = np.cumsum(gaps) - gaps[0]
    at_load = serve(arr_load, args.serve_workers)
    one = serve(arrivals, 1)
    rel = [abs(a["objective"] - b["objective"]) / abs(b["objective"]) for a, b in zip(mix, one)
           if a["status"] == 0 and b["status"] == 0]
    per_request = [{"n": p.n, "k": p.k, "nnz": p.nnz, "loss": p.loss, "lambda_frac": float(f),
                    "status": int(r["status"]), "iters": int(r["iters"]), "ms": 1000.0 * (r["end"] - r["start"])}
                   for p, f, r in zip(problems, fracs, mix)]
    stop = (f"relative duality gap <= {args.serve_tol_gap:g}" if args.serve_tol_gap > 0 else
            f"KKT <= {args.serve_tol:g} lambda")
    return {"per_request_saturated": per_request,
            "workload": f"config 5: {len(problems)} requests, "
                        f"{sum(p.nnz for p in problems) / 1e6:.0f}M nnz in total, FP32, {stop} per request, "
                        f"Thread-Greedy B=1024",
            "slots": args.serve_workers,
            "saturated": sat,
            "sustained": summary(at_load, rate),
            "one_at_a_time": summary(one, 200.0),
            "speedup_over_one_at_a_time": sat["solves_per_s"] / summary(one, 200.0)["solves_per_s"],
            "max_rel_objective_diff": max(rel) if rel else None}


def run_batch_step(args):
    """The batched Thread-Greedy step alone: config 4 (scaled by --path-scale),
    5 folds, every slot active (fold s mod 5, lambda = 0.05 lambda_max of
    the fold, w = 0), --warmup untimed then --steps timed steps (CUDA events
    on the library's stream)."""
    import torch

    from paper_1206_6409_gb300 import binding as gb

    gb.lib()
    prob = workloads.config4(args.path_loss, seed=0, scale=args.path_scale)
    fold = workloads.cv_folds(prob.n, PATH_FOLDS, seed=0)
    st = torch.cuda.current_stream()
    with gb.Batch(prob, fold=fold, nfolds=PATH_FOLDS, slots=args.batch_step, stream=st.cuda_stream) as b:
        b.set_params(variant="thread_greedy", blocks=args.path_blocks)
        for s in range(b.slots):
            h = s % PATH_FOLDS
            b.set_slot(s, h, 0.05 * b.lambda_max(h), None)
        b.iterate(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.iterate(args.steps, sync=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(1, args.steps)
        print(json.dumps({"metric": "batched Thread-Greedy step", "workload": prob.name, "slots": b.slots,
                          "blocks": args.path_blocks, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "us_per_solve_step": 1000.0 * ms / b.slots}), flush=True)


def run_reference(args):
    """The reference arm: the paper's method has no runnable implementation,
    so the OpenMP baseline (Section 4.2's design, FP64) runs the workload on
    the host's cores: one step = one Thread-Greedy iteration over the whole
    workload (stored values of the storage mode), continuing from the last."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    prob = load_problem(args.scale, args.precision)
    import oracle

    sp = oracle.stored_problem(prob, args.precision) if args.precision != "f64" else prob
    orc = oracle.Oracle(sp)
    lam = 0.05 * orc.lambda_max()
    orc.set_lambda(lam)
    info = host_info()
    s = oracle.OmpSolver(orc)
    s.iterate(args.warmup, B=args.blocks)
    t0 = time.perf_counter()
    _, nnz, _ = s.iterate(args.steps, B=args.blocks)
    el = time.perf_counter() - t0
    s.close()
    value = nnz / el
    line = {"impl": "reference", "metric": "nnz processed/s", "value": value, "unit": "nnz/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (WORKLOAD_DESC if args.scale >= 1.0 else f"scaled {args.scale}: {prob.name}")
                       + ("; binarized: every non-zero of column j is 1/sqrt(nnz_j)"
                          if args.precision == "binary" else ""),
                       "variant": "thread_greedy", "blocks": args.blocks, "precision": args.precision,
                       "oracle_arithmetic": "f64"},
            "cpu_baseline": {"kind": "oracle", "impl": "OpenMP Thread-Greedy (Section 4.2: static schedule, "
                                                       "atomic z), FP64", "cores": s.threads, "value": value,
                             "unit": "nnz/s", "same_config": True, **info,
                             "sample": f"{args.steps} Thread-Greedy iterations (B={args.blocks}) of the whole "
                                       f"workload after {args.warmup} warm-up iterations, {el:.1f} s on "
                                       f"{s.threads} threads"},
            "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _event_ms(fn, stream):
    """Device time (ms) of the work fn enqueues on `stream` (CUDA events)."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def time_to_target(args, gb, prob, val, lam, stream):
    """Time to a 1e-6 relative objective gap from w = 0 (reading 10).

    P* comes from a reference solve of the same problem (the stored values of
    the storage mode) in FP64 arithmetic: Thread-Greedy with the accept
    backoff, to KKT <= 1e-6 lambda or --ref-seconds.  The CPU-baseline leg
    certifies that point with the oracle (KKT violation and duality gap in
    FP64).  The timed run is the benchmark's own configuration from w = 0, with
    an objective check every --target-check iterations inside the clock."""
    import torch

    ref_val = stored_values_host(val, args.precision)
    q = gb.Problem(n=prob.n, k=prob.k, col_ptr=prob.col_ptr, row_idx=prob.row_idx, val=ref_val, y=prob.y,
                   loss="logistic", precision="f64", stream=stream.cuda_stream)
    q.set_lambda(lam)
    q.set_params(variant="thread_greedy", blocks=args.blocks, seed=0, tol_kkt=1e-6 * lam, max_iter=10_000_000,
                 check_every=20, timeout_s=args.ref_seconds)
    r = q.solve()
    w_ref = q.w()
    p_star, ref_kkt = q.objective()
    q.close()
    ref = {"objective": p_star, "kkt": ref_kkt, "kkt_over_lambda": ref_kkt / lam, "status": int(r.status),
           "iterations": int(r.iters), "seconds": r.seconds,
           "w_sha256": hashlib.sha256(np.ascontiguousarray(w_ref).tobytes()).hexdigest()[:16],
           "w_nonzeros": int(np.count_nonzero(w_ref)),
           "how": "FP64 Thread-Greedy (B=%d, accept backoff) on the stored values to KKT <= 1e-6 lambda or %g s"
                  % (args.blocks, args.ref_seconds)}
    p = gb.Problem(n=prob.n, k=prob.k, col_ptr=prob.col_ptr, row_idx=prob.row_idx, val=val, y=prob.y,
                   loss="logistic", precision=args.precision, stream=stream.cuda_stream)
    p.set_lambda(lam)
    p.set_params(variant=args.variant, blocks=args.blocks, seed=0)
    p.stats_reset()
    torch.cuda.synchronize()
    target = p_star * (1.0 + 1e-6)
    t0 = time.perf_counter()
    iters, reached, obj = 0, False, None
    while iters < args.target_max_iter and time.perf_counter() - t0 < 60.0:
        p.iterate(args.target_check, sync=False)
        iters += args.target_check
        obj, _ = p.objective()
        if obj <= target:
            reached = True
            break
    el = time.perf_counter() - t0
    st = p.stats()
    p.close()
    out = {"seconds": el if reached else None, "iterations": iters, "reached": reached, "rel_gap": 1e-6,
           "objective": obj, "rel_gap_at_end": (obj - p_star) / p_star if obj is not None else None,
           "check_every": args.target_check, "updates": int(st.updates),
           "updates_per_s": st.updates / el if el > 0 else None, "p_star": p_star, "reference": ref}
    return out, w_ref


def _step_leg(gb, prob, val, precision, lam, stream, steps, variant="thread_greedy", blocks=1024, warm=3,
              extra=None):
    """Times `steps` iterations of one configuration on config 2 (CUDA events
    on the library's stream, after `warm` untimed ones)."""
    p = gb.Problem(n=prob.n, k=prob.k, col_ptr=prob.col_ptr, row_idx=prob.row_idx, val=val, y=prob.y,
                   loss="logistic", precision=precision, stream=stream.cuda_stream)
    try:
        p.set_lambda(lam)
        out = {}
        if extra:
            out.update(extra(p))
        p.set_params(variant=variant, blocks=blocks, seed=0)
        p.iterate(warm, sync=False)
        gb.gencd_profile_reset(p.h)
        p.stats_reset()
        gb.gencd_profile_enable(p.h, True)
        ms = _event_ms(lambda: p.iterate(steps, sync=False), stream)
        st = p.stats()
        prof = {name: gb.gencd_profile_read(p.h, name) for name in gb.KERNELS}
        gb.gencd_profile_enable(p.h, False)
        out.update({"ms_per_step": ms / steps, "us_per_iteration": 1000.0 * ms / steps,
                    "nnz_per_s": st.nnz_processed / (ms / 1000.0), "updates_per_s": st.updates / (ms / 1000.0),
                    "updates_per_step": st.updates / steps, "steps": steps,
                    "kernel_ms_per_call": {k: v[0] / v[2] for k, v in prof.items() if v[2]}})
        return out, prof
    finally:
        p.close()


def leg_storage_modes(args, gb, prob, stream):
    """Config 2, one Thread-Greedy step in the storage modes the headline does
    not run: ms/step, nnz/s and the streaming propose's roofline fraction."""
    out = {}
    peak, _ = measured_peak()
    for mode in ("f32", "f64", "bf16", "binary"):
        if mode == args.precision:
            continue
        src = workloads.binarized(prob) if mode == "binary" else prob
        val = src.val if mode == "f64" else src.val.astype(np.float32)
        try:
            lm_probe = gb.Problem(n=src.n, k=src.k, col_ptr=src.col_ptr, row_idx=src.row_idx, val=val, y=src.y,
                                  loss="logistic", precision=mode, stream=stream.cuda_stream)
            lam = 0.05 * lm_probe.lambda_max()
            lm_probe.close()
            r, prof = _step_leg(gb, src, val, mode, lam, stream, args.leg_steps, blocks=args.blocks)
            sv = VALUE_BYTES[mode]
            byts = src.nnz * (4 + sv) + 8 * (src.k + 1) + 8 * src.k + (4 * src.k if sv == 0 else 0)
            pa_ms, _, pa_n = prof["propose_all"]
            if pa_n:
                r["roofline"] = {"achieved_gbs": byts / (pa_ms / pa_n / 1000.0) / 1e9,
                                 "frac": byts / (pa_ms / pa_n / 1000.0) / 1e9 / peak,
                                 "algorithmic_bytes_per_launch": byts, "launch_ms": pa_ms / pa_n}
            out[mode] = r
        except Exception as e:  # noqa: BLE001 -- reported, the headline still prints
            out[mode] = {"error": f"{type(e).__name__}: {e}"}
    return out


def leg_variants(args, gb, prob, val, lam, stream):
    """Config 2 in the benchmark's storage mode with Shotgun (Table 2; P*
    columns per iteration after the power iteration): time per iteration,
    nnz/s, updates/s and the one-time cost.  (Coloring is timed on config 1:
    the distance-2 colouring of this workload is impractical.)"""
    import torch

    out = {}

    def pstar(p):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rho, ps, it = p.spectral_radius()
        torch.cuda.synchronize()
        return {"setup_s": time.perf_counter() - t0, "rho": rho, "P_star": int(ps), "power_iterations": int(it)}

    out["coloring"] = {"skipped": "the distance-2 colouring of this workload visits sum_i deg(i)^2 ~ 4e10 "
                                  "neighbour pairs per round (rows hold ~200 entries and columns up to 50,000); "
                                  "Coloring runs on config 1 (legs.config1)"}
    for name, variant, extra, steps in (("shotgun", "shotgun", pstar, 200),):
        try:
            out[name], _ = _step_leg(gb, prob, val, args.precision, lam, stream, steps, variant=variant,
                                     extra=extra)
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def leg_config1(args, gb, stream):
    """Config 1 (n = 2,000, k = 5,000, +-1 values, FP64), both losses,
    lambda = 0.01 lambda_max: Shotgun at P* and Coloring solved from w = 0 to
    KKT <= 1e-9 (latency: wall time, iterations, us per iteration, nnz/s)."""
    out = {}
    for loss in ("logistic", "squared"):
        prob = workloads.config1(loss)
        for variant in ("shotgun", "coloring"):
            try:
                with gb.Problem(prob, precision="f64", stream=stream.cuda_stream) as p:
                    p.set_lambda(0.01 * p.lambda_max())
                    if variant == "shotgun":
                        p.spectral_radius()
                    else:
                        p.color()
                    # Coloring takes about 1.5e6 iterations to 1e-9 on the logistic problem: capped
                    p.set_params(variant=variant, tol_kkt=1e-9, max_iter=300_000 if variant == "coloring" else 5_000_000,
                                 check_every=200, seed=0)
                    p.solve()  # warm-up (kernel loading), then the same solve from w = 0
                    p.set_w(np.zeros(prob.k))
                    p.set_iteration(0)
                    r = p.solve()
                out[f"{variant}_{loss}"] = {"status": int(r.status), "seconds": r.seconds, "iterations": int(r.iters),
                                            "us_per_iteration": 1e6 * r.seconds / max(1, r.iters),
                                            "nnz_per_s": r.nnz_processed / r.seconds if r.seconds > 0 else None,
                                            "updates_per_s": r.updates / r.seconds if r.seconds > 0 else None,
                                            "objective": r.objective, "kkt": r.kkt}
            except Exception as e:  # noqa: BLE001
                out[f"{variant}_{loss}"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_gencd(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1206_6409_gb300 import binding as gb

    gb.lib()
    prob = load_problem(args.scale, args.precision)
    stream = torch.cuda.current_stream()
    val = prob.val if args.precision == "f64" else prob.val.astype(np.float32)

    # ---- device-resident arm ----------------------------------------------
    p = gb.Problem(n=prob.n, k=prob.k, col_ptr=prob.col_ptr, row_idx=prob.row_idx, val=val, y=prob.y,
                   loss="logistic", precision=args.precision, stream=stream.cuda_stream)
    lam = 0.05 * p.lambda_max()
    p.set_lambda(lam)
    p.set_params(variant=args.variant, blocks=args.blocks, seed=0)
    if args.propose_split >= 0:
        gb.gencd_set_propose_schedule(p.h, args.propose_split)
    split, tuned = gb.gencd_propose_schedule(p.h)
    schedule = {"fused_split": split, "candidates_ms": tuned,
                "form": "separate light and slab kernels" if split == 0 else
                f"one kernel, {split} of 32 warps per SM start on the row slabs"}
    for _ in range(args.warmup):
        p.iterate(1, sync=False)
    torch.cuda.synchronize()
    gb.gencd_profile_reset(p.h)
    p.stats_reset()
    gb.gencd_profile_enable(p.h, True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        p.iterate(1, sync=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    st = p.stats()
    prof = {name: gb.gencd_profile_read(p.h, name) for name in gb.KERNELS}
    gb.gencd_profile_enable(p.h, False)
    final_obj, final_kkt = p.objective()  # after the timed region
    w_nonzeros = int(np.count_nonzero(p.w()))
    launches = int(sum(v[1] for v in prof.values()))
    nnz_done = int(st.nnz_processed)
    (ms,), (nnz_total,) = reduce_over_ranks([ms], [nnz_done], "cuda")
    value = nnz_total / (ms / 1000.0)

    # roofline of the dominant kernel: the streaming propose's pass over X
    # (k_propose_fused, or the two separate passes when the autotuner keeps
    # them), with what it must move as its algorithmic bytes: the X stream
    # (row index + stored value per non-zero; u is L2-resident) and the
    # gradient it writes (one g_j per column, FP32 or FP64); the family (every
    # kernel of the propose over all columns) counts a column pointer and an
    # FP64-sized gradient per column instead
    pa_ms, _, pa_n = prof["propose_all"]  # one timed invocation of the family per step
    sv = VALUE_BYTES[args.precision]
    bytes_per_launch = prob.nnz * (4 + sv) + 8 * (prob.k + 1) + 8 * prob.k + (4 * prob.k if sv == 0 else 0)
    family_achieved = bytes_per_launch / (pa_ms / pa_n / 1000.0) / 1e9 if pa_n else None
    g_bytes = 8 if args.precision == "f64" else 4
    x_bytes = prob.nnz * (4 + sv) + (4 * prob.k if sv == 0 else 0) + g_bytes * prob.k
    if prof["propose_fused"][2]:
        dom_name, (dom_ms, _, dom_n) = "k_propose_fused", prof["propose_fused"]
    else:
        dom_name = "k_propose_light_runs + k_propose_slabs"
        dom_ms = prof["propose_light"][0] + prof["propose_slabs"][0]
        dom_n = max(prof["propose_light"][2], prof["propose_slabs"][2])
    achieved = x_bytes / (dom_ms / dom_n / 1000.0) / 1e9 if dom_n else None
    peak, peak_kind = measured_peak()
    csrc = os.path.join(ROOT, "paper_1206_6409_gb300", "csrc")
    traffic, src_hash = recorded_traffic([os.path.join(csrc, f) for f in ("kernels_propose.cu", "propose_plan.cu")],
                                         args.precision)
    p.close()
    del p

    # ---- end-to-end arm through the C ABI from pinned host buffers ---------
    e2e = None
    if args.e2e_steps > 0:
        pin = {}
        for name, a in (("col_ptr", prob.col_ptr), ("row_idx", prob.row_idx), ("val", val), ("y", prob.y)):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            pin[name] = t.numpy()
        h2d = sum(a.nbytes for a in pin.values())
        d2h = 64  # objective, KKT and the work counters
        torch.cuda.synchronize()
        t_e2e = 0.0
        nnz_e2e = 0
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q = gb.Problem(n=prob.n, k=prob.k, loss="logistic", precision=args.precision,
                           stream=stream.cuda_stream, **pin)
            q.set_lambda(0.05 * q.lambda_max())
            q.set_params(variant=args.variant, blocks=args.blocks, seed=0)
            q.stats_reset()
            q.iterate(1, sync=False)
            r = q.stats()
            q.close()
            el = time.perf_counter() - t0
            if i > 0:  # the first step is a warm-up
                t_e2e += el
                nnz_e2e += int(r.nnz_processed)
        e2e = {"value": nnz_e2e / t_e2e, "unit": "nnz/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h,
               "ms_per_step": 1000.0 * t_e2e / args.e2e_steps}
        (t_max,), (nnz_sum,) = reduce_over_ranks([t_e2e], [nnz_e2e], "cuda")
        e2e["value"] = nnz_sum / t_max

    # ---- time to a 1e-6 relative objective gap from w = 0 -------------------
    ttt, w_ref = None, None
    if args.target_check > 0:
        ttt, w_ref = time_to_target(args, gb, prob, val, lam, stream)

    # ---- the other storage modes and variants of config 2, config 1 --------
    legs = {}
    if args.legs:
        legs["storage_modes"] = leg_storage_modes(args, gb, prob, stream)
        legs["variants"] = leg_variants(args, gb, prob, val, lam, stream)
        legs["config1"] = leg_config1(args, gb, stream)

    path = None
    if args.path:
        try:
            path = run_path(args, gb, stream)
        except Exception as e:  # reported, not fatal: the headline line still prints
            path = {"error": f"{type(e).__name__}: {e}"}

    serve = None
    if args.serve:
        try:
            serve = run_serve(args, gb)
        except Exception as e:  # reported, not fatal
            serve = {"error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        sp = prob if args.precision == "f64" else oracle.stored_problem(prob, args.precision)
        cpu, cert = cpu_baseline_leg(sp, lam, args.blocks, w_ref)
        if ttt is not None:
            ttt["p_star_certificate"] = cert

    if rank == 0:
        line = {
            "metric": "nnz processed/s", "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": (WORKLOAD_DESC if args.scale >= 1.0 else f"scaled {args.scale}: {prob.name}")
                       + ("; binarized: every non-zero of column j is 1/sqrt(nnz_j)"
                          if args.precision == "binary" else ""),
                       "variant": args.variant, "blocks": args.blocks, "precision": args.precision,
                       "nnz": prob.nnz, "n": prob.n, "k": prob.k,
                       "l2": "inputs larger than L2: each step streams all of X (%.2f GB)" % (bytes_per_launch / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "traffic": traffic,
                         "algorithmic_bytes_per_launch": x_bytes,
                         "launch_ms": dom_ms / dom_n if dom_n else None, "source_sha256": src_hash,
                         "family": {"kernels": "every kernel of the propose over all columns", "achieved": family_achieved,
                                    "frac": family_achieved / peak if family_achieved else None,
                                    "algorithmic_bytes_per_launch": bytes_per_launch,
                                    "launch_ms": pa_ms / pa_n if pa_n else None}},
            "propose_schedule": schedule,
            "kernel_ms_per_call": {k: v[0] / v[2] for k, v in prof.items() if v[2]},
            "kernel_launches": {k: v[1] for k, v in prof.items() if v[1]},
            "gpu_launches": launches,
            "updates_per_step": st.updates / args.steps,
            "updates_per_s": st.updates / (ms / 1000.0),
            "time_to_1e-6": ttt,
            "legs": legs,
            "objective": final_obj, "kkt": final_kkt, "w_nonzeros": w_nonzeros,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "regularisation_path": path,
            "serving": serve,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.batch_step > 0:
        run_batch_step(args)
    else:
        run_gencd(args)


if __name__ == "__main__":
    main()
