"""Benchmark: batched MPC QPs solved to relative KKT 1e-6 on B300, QP solves/sec.

Workload (default ``--workload mpc_batch``): 4,096 linear-MPC QPs, horizon
T ~ U{10..50}, 12 states / 4 inputs (n = 16T, m = 12T), solved to relative KKT
1e-6 by one persistent launch of the PDHCG-II kernel (pdhcg_solve_batch), FP32
matrix values, double-float vectors and FP64 reductions.  Also timed: the plain
one-at-a-time solver on a sample of the same instances, the end-to-end path
through the public API (problem upload + device setup + solve + result
download), and the FP64 CPU oracle on a sample (cpu_baseline).

``--impl reference`` times the CPU oracle alone on the same workload and metric.
Multi-GPU (torchrun): every rank solves its own 4,096 instances (weak scaling,
no collective in the data path; one barrier and a max over ranks for timing).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_23967_b300 import workloads as W  # noqa: E402

METRIC = "QP solves/sec and SpMV HBM GB/s at rel. KKT 1e-6, batched/served vs plain"
UNIT = "solves/s"
EPS = 1e-6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mpc_batch", choices=["mpc_batch"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: each rank solves its own --count instances; strong: the ranks split one "
                         "batch of --count instances by the work-weighted partition")
    ap.add_argument("--precision", default="dfloat", choices=["dfloat", "mixed", "fp64", "fp32"])
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=96)
    ap.add_argument("--ablation", default=None, choices=["inner-tolerance", "inner-solver"],
                    help="instead of the benchmark: the adaptive inner tolerance (Sec. 3.3) against fixed ones")
    ap.add_argument("--large-iters", type=int, default=128,
                    help="PDHG steps timed on the large sparse QP (n=2e6); 0 skips it")
    ap.add_argument("--large-n", type=int, default=2_000_000,
                    help="variables of that QP (m = n/2); smaller values are for profiling captures")
    ap.add_argument("--large-form", default="auto", choices=["auto", "pipeline", "persistent"],
                    help="how that QP runs: the library's choice, the pipeline graph, or the persistent kernel")
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[200.0, 2000.0],
                    help="Poisson arrival rates (requests/s) of the serving traces; none skips serving")
    ap.add_argument("--serve-eps", type=float, nargs="*", default=[1e-4, 1e-6])
    ap.add_argument("--serve-requests", type=int, default=120, help="arrivals per serving trace")
    ap.add_argument("--serve-plain", type=int, default=16, help="requests the plain solver times per trace")
    ap.add_argument("--serve-slots", type=int, default=2 * 148, help="concurrent solves of the serving loop")
    ap.add_argument("--serve-mpc-rate", type=float, default=3000.0,
                    help="arrival rate of a 4 s trace of MPC requests only, run with the serving traces "
                         "(0: skip; an empty --serve-rates skips all serving)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the row layout and launch shape with pdhcg_autotune (batch: on a 512-instance "
                         "sample; large sparse QP: on the instance) before timing")
    ap.add_argument("--whole-eps", type=float, nargs="*", default=[1e-4, 1e-6],
                    help="tolerances of the whole-solve legs (portfolio and large sparse QP)")
    ap.add_argument("--whole-large-limit", type=float, default=20.0,
                    help="device-time limit (s) of each large sparse QP solve; 0 skips it")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def instances(count, rank, world=1, scaling="weak"):
    """The instances rank r solves.  weak: its own ``count`` instances (seed
    1000 r), so per-GPU work is fixed as ranks are added.  strong: rank r's
    share of one fixed batch of ``count`` instances, split by the greedy
    work-weighted partition (every rank computes the same split)."""
    if scaling == "weak":
        return W.mpc_batch(count=count, seed=1000 * rank)
    from paper_2602_23967_b300 import partition as PT
    qps = W.mpc_batch(count=count, seed=0)
    parts = PT.partition([PT.work_estimate(q, diagonal_q=True) for q in qps], world)
    return [qps[i] for i in parts[rank]]


def config_of(args):
    """The workload description both arms print."""
    per = "per GPU" if args.scaling == "weak" else "split over the GPUs by a work-weighted partition"
    return {"workload": f"mpc_batch: {args.count} MPC QPs {per} (T~U{{10..50}}, 12 states, "
                        f"4 inputs, n=16T, m=12T), rel. KKT {EPS:g}, one persistent launch",
            "l2": "inputs larger than L2 (whole batch ~0.5 GB)", "precision": args.precision}


def max_over_ranks(value, world, device="cpu"):
    """Largest ``value`` over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, count, steps, total_ms, scaling="weak"):
    """Whole-job solves/s: every rank solved ``count`` instances per step
    (weak), or all ranks together solved ``count`` per step (strong)."""
    per_step = world * count if scaling == "weak" else count
    return per_step * steps / (total_ms * 1e-3)


def input_bytes(qp):
    b = qp.A.nnz * 12 + (qp.m + 1) * 8 + 5 * 8 * qp.n + 2 * 8 * qp.m
    if qp.Q is not None:
        b += qp.Q.nnz * 12 + (qp.n + 1) * 8
    return b


def algorithmic_bytes(qp, iterations, mat_bytes=4, idx_bytes=4, vec_bytes=8):
    """Algorithmic bytes of the batched kernel for one instance (diagonal Q, so no inner solver).

    Per PDHG step: A x and A^T y streamed once (2 Z (v + i)), row pointers
    (4 (n + m + 2)), vectors s (10 n + 7 m): Phase I reads x, c, lv, uv, diag Q,
    anchor and gathers y, writes x+, xbar, x_new; Phase II gathers xbar, reads
    y, lc, uc, anchor and writes y+, y_new.  Every 64 steps the check adds one
    pass over A (two gathers), A^T and Q plus 8 n + 6 m vector reads."""
    Z = qp.A.nnz
    W_ = qp.Q.nnz if qp.Q is not None else 0
    n, m = qp.n, qp.m
    per_it = 2 * Z * (mat_bytes + idx_bytes) + 4 * (n + m + 2) + vec_bytes * (10 * n + 7 * m)
    per_check = (2 * Z + W_) * (mat_bytes + idx_bytes) + vec_bytes * (8 * n + 6 * m)
    return iterations * per_it + (iterations // 64) * per_check


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(qps, sample, time_budget_s=25.0):
    """FP64 CPU oracle (single thread) on the first instances of the workload."""
    import oracle
    oracle.build()
    t0 = time.time()
    results = []
    for q in qps[:sample]:
        x, y, r = oracle.solve(q, oracle.default_params(eps_tol=EPS))
        results.append(r)
        if time.time() - t0 > time_budget_s:
            break
    dt = time.time() - t0
    return len(results) / dt, results, dt


# DRAM traffic of the batched solve kernel from one ncu capture on 512 instances
# (dram__bytes_read.sum + dram__bytes_write.sum), per instance; valid only for the
# kernel sources it was taken on (hash below), else the roofline reports null.
TRAFFIC_CAPTURE = {"bytes": 1_848_600_320 + 1_397_771_520, "instances": 512,
                   "sources_sha256": "15bbaee1c95199a85b19b9658ebd977f69aeef56e7b08a80db8e95cca51dbcaf",
                   "summary": "profiles/solve_kernel_mpc_batch512_dram.md"}
KERNEL_SOURCES = ("solve_kernel.cuh", "device_common.cuh", "dfloat.cuh", "launch.h", "kernels_impl.cuh",
                  "pdhcg_internal.h", "kernels_dfloat.cu")


def code_of(text):
    """C/C++/CUDA source with comments and blank lines removed, so that the hash
    below follows the code only (string literals in kernel sources hold no
    comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_sources_sha256(read=None):
    """SHA-256 over the code (comments stripped) of the solve kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_2602_23967_b300", "csrc", name)) as f:
                text = f.read()
        else:
            text = read(name)
        h.update(code_of(text).encode())
    return h.hexdigest()


def traffic_per_launch(count):
    """Measured DRAM bytes scaled to ``count`` instances, or None if the kernel changed."""
    cap = TRAFFIC_CAPTURE
    if cap["sources_sha256"] != kernel_sources_sha256():
        return None
    return cap["bytes"] * count / cap["instances"]


def fp64_kkt(qp, x, y):
    """Relative KKT residuals of Sec. 4.2 of a returned (x, y), from the problem
    data in FP64 (scipy products), independently of the device's evaluation:
    max(r_primal, r_dual, r_gap)."""
    Ax = qp.A @ x
    ATy = qp.A.T @ y if qp.m else np.zeros(qp.n)
    Qx = qp.Q @ x if qp.Q is not None else np.zeros(qp.n)
    fin = lambda v: np.abs(v[np.isfinite(v)])  # noqa: E731
    bnd = np.concatenate([fin(qp.lc), fin(qp.uc)])
    r_p = np.max(np.abs(Ax - np.clip(Ax, qp.lc, qp.uc)), initial=0.0) / (1.0 + np.max(bnd, initial=0.0))
    r = Qx + qp.c + ATy
    lf, uf = np.isfinite(qp.lv), np.isfinite(qp.uv)
    rh = np.where(lf & uf, r, np.where(lf, np.maximum(r, 0.0), np.where(uf, np.minimum(r, 0.0), 0.0)))
    r_d = np.max(np.abs(r - rh), initial=0.0) / (
        1.0 + max(np.max(np.abs(Qx), initial=0.0), np.max(np.abs(ATy), initial=0.0), np.max(np.abs(qp.c), initial=0.0)))

    def p(z, lo, hi):  # p(z; l, u) = u^T z+ - l^T z-, zero entries contribute 0
        pos, neg = z > 0, z < 0
        return float(np.sum(hi[pos] * z[pos]) + np.sum(lo[neg] * z[neg]))

    xQx, cx = float(x @ Qx), float(qp.c @ x)
    pr, py = p(-rh, qp.lv, qp.uv), p(y, qp.lc, qp.uc)
    r_g = abs(xQx + cx + pr + py) / (1.0 + max(abs(0.5 * xQx + cx), abs(0.5 * xQx + pr + py)))
    return max(r_p, r_d, r_g)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def large_bytes(qp, iterations, inner, mat_bytes=4, idx_bytes=4, vec_bytes=8, k_eval=64):
    """Algorithmic bytes of `iterations` PDHG steps with `inner` BB/CG steps on a
    QP with a general Q: per PDHG step A^T y, Q x and A xbar streamed once plus
    s (10 n + 7 m) of vectors; per inner step one pass over Q plus 6 s n; per
    check (every k_eval steps) A twice, A^T and Q once, s (8 n + 6 m)."""
    Z, Wq, n, m = qp.A.nnz, qp.Q.nnz, qp.n, qp.m
    v = mat_bytes + idx_bytes
    per_it = (2 * Z + Wq) * v + 4 * (2 * n + m + 3) + vec_bytes * (10 * n + 7 * m)
    per_inner = Wq * v + 4 * (n + 1) + 6 * vec_bytes * n
    per_check = (3 * Z + Wq) * v + vec_bytes * (8 * n + 6 * m)
    return iterations * per_it + inner * per_inner + (iterations // k_eval) * per_check


def large_instance_leg(args, stream, peak_gbs):
    """One large sparse QP (n = 2e6, m = 1e6, ~10 nnz/row in Q, ~8 in A with
    power-law column degrees) on a multi-CTA group: device time of a fixed
    number of PDHG steps, and the algorithmic bytes they stream."""
    import torch
    from paper_2602_23967_b300 import pdhcg
    qp = W.large_sparse_qp(n=args.large_n, m=args.large_n // 2, seed=0)
    prm = pdhcg.default_params(precision=args.precision, eps_tol=1e-12, max_iter=args.large_iters,
                               pipeline={"auto": 0, "pipeline": 1, "persistent": -1}[args.large_form])
    tune = None
    if args.autotune:
        prm, tune = pdhcg.autotune([qp], prm, stream=stream.cuda_stream)
    p = pdhcg.Problem(qp, prm, stream=stream.cuda_stream)
    try:
        x = torch.empty(qp.n, dtype=torch.float64, device="cuda")
        y = torch.empty(qp.m, dtype=torch.float64, device="cuda")
        p.solve_dev(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = p.solve_dev(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        p.close()
    mb, vb = {"fp64": (8, 8), "fp32": (4, 4)}.get(args.precision, (4, 8))
    alg = large_bytes(qp, r["iterations"], r["inner_iterations"], mat_bytes=mb, vec_bytes=vb)
    gbs = alg / (ms * 1e-3) / 1e9
    forms = {0: "one CTA", 1: "persistent multi-CTA group", 2: "pipeline graph (one kernel per phase)"}
    return {"workload": f"large sparse QP n={qp.n}, m={qp.m}, nnz(Q)={qp.Q.nnz}, nnz(A)={qp.A.nnz}, "
                        f"{r['iterations']} PDHG steps ({r['inner_iterations']} BB steps)",
            "form": forms.get(r["form"], r["form"]),
            "us_per_step": ms * 1e3 / r["iterations"], "algorithmic_bytes": alg,
            "achieved_gbs": gbs, "frac_of_hbm_peak": gbs / peak_gbs, "autotune": tune,
            "calibration": gather_calibration(qp.Q, stream)}


def gather_calibration(Q, stream, reps=20):
    """Library reference points on the same Q (2e7 nonzeros at uniformly random
    columns), timed with CUDA events: torch.index_select of an 8-byte entry per
    nonzero from an n-entry table (the random-gather rate of the device when the
    table sits in L2, plus the index and output streams) and the cuSPARSE SpMV
    behind torch.mv on a CSR tensor, FP32 and FP64.  Not part of the solver."""
    import warnings

    import torch
    dev = torch.device("cuda")
    crow = torch.from_numpy(Q.indptr.astype(np.int32)).to(dev)
    col = torch.from_numpy(Q.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(Q.data).to(dev)
    n, nnz = Q.shape[0], Q.nnz

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e3

    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        out = {}
        tab = torch.randn(n, dtype=torch.float64, device=dev)
        idx = col.long()
        us = timed(lambda: torch.index_select(tab, 0, idx))
        out["index_select_8B_us"] = us
        out["random_gathers_per_s"] = nnz / (us * 1e-6)
        for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
            M = torch.sparse_csr_tensor(crow, col, val.to(dt), size=(n, n))
            x = torch.randn(n, dtype=dt, device=dev)
            out[f"cusparse_{name}_spmv_us"] = timed(lambda: torch.mv(M, x))
        del tab, idx
    out["note"] = ("reference points only: the solver's Q product is its own kernel; per PDHG step it "
                   "runs about (1 + BB steps per PDHG step) of them")
    return out


def serve_trace(prm, stream, trace, qps, slots, drain_s=90.0):
    """Replays an arrival trace against the serving loop: each request is
    submitted at its arrival time through pdhcg_submit and collected with
    pdhcg_poll; latency is the server's submit-to-ready wall time."""
    from paper_2602_23967_b300 import pdhcg
    srv = pdhcg.Server(hbm_budget_bytes=100 << 30, max_slots=slots, params=prm, stream=stream)
    t_sub, out, pending, kinds = {}, {}, [], {}
    try:
        t0 = time.perf_counter()
        i = 0
        while i < len(trace) or pending:
            now = time.perf_counter() - t0
            while i < len(trace) and trace[i][0] <= now:
                tk = srv.submit(qps[i])
                t_sub[tk] = time.perf_counter() - t0
                kinds[tk] = trace[i][1]
                pending.append(tk)
                i += 1
            still = []
            for tk in pending:
                r = srv.poll(tk)
                if r is None:
                    still.append(tk)
                else:
                    out[tk] = r[2]
            pending = still
            if now > trace[-1][0] + drain_s:
                break
            time.sleep(0.0005)
        st = srv.stats()
    finally:
        srv.close()
    lat = np.array([out[tk]["latency_seconds"] for tk in out])
    ready = np.array([t_sub[tk] + out[tk]["latency_seconds"] for tk in out])
    span = float(ready.max() - min(t_sub.values())) if len(out) else float("nan")
    by_kind = {}
    for kind in sorted(set(kinds.values())):
        lk = np.array([out[tk]["latency_seconds"] for tk in out if kinds[tk] == kind])
        # device span of the solve (first step to last, pauses included) and the rest of
        # the latency (queue, admission, setup, retirement)
        sk = np.array([out[tk]["solve_seconds"] for tk in out if kinds[tk] == kind])
        by_kind[kind] = {"requests": sum(1 for v in kinds.values() if v == kind), "completed": int(len(lk)),
                         "latency_p50_ms": float(np.percentile(lk, 50) * 1e3) if len(lk) else None,
                         "latency_p99_ms": float(np.percentile(lk, 99) * 1e3) if len(lk) else None,
                         "solve_span_p50_ms": float(np.percentile(sk, 50) * 1e3) if len(sk) else None,
                         "wait_p50_ms": float(np.percentile(lk - sk, 50) * 1e3) if len(sk) else None}
    statuses = [r["status_name"] for r in out.values()]
    return {"requests": len(trace), "completed": len(out),
            "optimal": statuses.count("OPTIMAL"), "primal_infeasible": statuses.count("PRIMAL_INFEASIBLE"),
            "solves_per_s": len(out) / span if len(out) else None,
            "latency_p50_ms": float(np.percentile(lat, 50) * 1e3) if len(out) else None,
            "latency_p99_ms": float(np.percentile(lat, 99) * 1e3) if len(out) else None,
            "latency_max_ms": float(lat.max() * 1e3) if len(out) else None,
            "by_kind": by_kind, "launches": st["launches"],
            "scheduler_seconds": {"admit": st["admit_seconds"], "slices": st["slice_seconds"],
                                  "retire": st["retire_seconds"]}}


def plain_sample(prm, stream, qps):
    """The plain one-at-a-time GPU solver (pdhcg_solve_dev per problem) on qps: solves/s."""
    import torch
    from paper_2602_23967_b300 import pdhcg
    probs = [pdhcg.Problem(q, prm, stream=stream) for q in qps]
    try:
        xo = torch.empty(max(p.n for p in probs), dtype=torch.float64, device="cuda")
        yo = torch.empty(max(max(p.m for p in probs), 1), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.time()
        for p in probs:
            p.solve_dev(xo, yo)
        torch.cuda.synchronize()
        return len(probs) / (time.time() - t0)
    finally:
        for p in probs:
            p.close()


def serving_leg(args, stream):
    """The serving workload: Poisson arrivals at each rate of --serve-rates of the
    request mix (70 % MPC, 25 % random QPs with n ~ U{1e3..1e5}, 2 % of them
    primal infeasible, 5 % factor-model QPs with n = 1e5), the first
    --serve-requests arrivals of each trace, served to each tolerance of
    --serve-eps; beside each, the plain one-at-a-time solver on the first
    --serve-plain requests of the same trace."""
    from paper_2602_23967_b300 import pdhcg
    rows = []
    for rate in args.serve_rates:
        trace = W.serving_trace(rate_per_s=rate, duration_s=1e9, seed=7, max_requests=args.serve_requests)
        qps = [W.build_request(k, sd, n) for _, k, sd, n in trace]
        for eps in args.serve_eps:
            prm = pdhcg.default_params(precision=args.precision, eps_tol=eps, time_limit_s=60.0)
            row = {"arrival_rate_per_s": rate, "eps": eps}
            row.update(serve_trace(prm, stream, trace, qps, args.serve_slots))
            if args.serve_plain > 0:
                plain = plain_sample(prm, stream, qps[: args.serve_plain])
                row["plain_solves_per_s"] = plain
                row["plain_sample"] = f"first {min(args.serve_plain, len(qps))} requests of the trace"
                if row["solves_per_s"]:
                    row["served_vs_plain"] = row["solves_per_s"] / plain
            rows.append(row)
    mpc_only = None
    if args.serve_mpc_rate > 0:
        # the serving loop's capacity on small requests: a 4 s trace of MPC QPs only
        trace = W.serving_trace(rate_per_s=args.serve_mpc_rate, duration_s=4.0, seed=7, mix=(1.0, 0.0, 0.0))
        qps = [W.build_request(k, sd, n) for _, k, sd, n in trace]
        prm = pdhcg.default_params(precision=args.precision, eps_tol=EPS, time_limit_s=60.0)
        mpc_only = {"arrival_rate_per_s": args.serve_mpc_rate, "eps": EPS, "duration_s": 4.0}
        mpc_only.update(serve_trace(prm, stream, trace, qps, args.serve_slots))
        mpc_only.pop("by_kind", None)
    return {"mix": "70 % MPC (T~U{10..50}), 25 % random QPs n~U{1e3..1e5} (~10 nnz/row, 2 % primal "
                   "infeasible), 5 % factor-model QPs n=1e5", "hbm_budget_gb": 100, "max_slots": args.serve_slots,
            "slice": "10 ms of device time per slice; MPC-sized requests on pool CTAs, larger ones on "
                     "multi-CTA groups in a cooperative launch of their own",
            "traces": rows, "mpc_only": mpc_only}


def whole_solve_leg(args, stream):
    """Whole solves of the factor-model portfolio QP (n = 1e5 + 1e3) and the
    large sparse QP (n = 2e6, m = 1e6) to each tolerance of --whole-eps, one
    handle each (pdhcg_create + pdhcg_solve_dev), with the FP64 KKT of the
    returned point evaluated on the host from the problem data."""
    import torch
    from paper_2602_23967_b300 import pdhcg
    rows = []
    # the large sparse QP does not reach 1e-4 within its limit, so it runs at
    # the loosest tolerance only (iterations/s and the KKT it reached)
    cases = [("factor_portfolio n=1e5+1e3, k=1e3", lambda: W.factor_portfolio(seed=0), 60.0, args.whole_eps),
             ("large_sparse_qp n=2e6, m=1e6", lambda: W.large_sparse_qp(seed=0), args.whole_large_limit,
              sorted(args.whole_eps)[-1:])]
    for name, make, limit, eps_list in cases:
        if limit <= 0:
            continue
        qp = make()
        x = torch.empty(qp.n, dtype=torch.float64, device="cuda")
        y = torch.empty(max(qp.m, 1), dtype=torch.float64, device="cuda")
        for eps in eps_list:
            prm = pdhcg.default_params(precision=args.precision, eps_tol=eps, time_limit_s=limit)
            t0 = time.time()
            p = pdhcg.Problem(qp, prm, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t_create = time.time() - t0
            try:
                r = p.solve_dev(x, y)
            finally:
                p.close()
            xs, ys = x.cpu().numpy(), y[: qp.m].cpu().numpy()
            k = fp64_kkt(qp, xs, ys)
            rows.append({"workload": name, "eps": eps, "status": r["status_name"], "iterations": r["iterations"],
                         "inner_iterations": r["inner_iterations"], "solve_s": r["solve_seconds"],
                         "create_s": t_create,
                         "solves_per_s": 1.0 / r["solve_seconds"] if r["status_name"] == "OPTIMAL" else 0.0,
                         "iterations_per_s": r["iterations"] / r["solve_seconds"],
                         "kkt_fp64": k, "objective": r["primal_obj"], "form": r["form"]})
    return rows


def _oracle_solve_one(qp):
    """One full FP64 oracle solve (runs in a spawned worker process)."""
    import oracle
    _, _, r = oracle.solve(qp, oracle.default_params(eps_tol=EPS))
    return r["status_name"]


def run_reference(args):
    """The FP64 C oracle on the host's cores: one solve per worker process at a
    time over consecutive instances of the same workload; each step is a
    bounded sample of 4 instances per core."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    qps = instances(args.count, 0)
    per_step = min(len(qps), 4 * cores)
    vals, t_all, done, off = [], 0.0, 0, 0
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_solve_one, qps[:cores], chunksize=1)
        for _ in range(args.steps):
            batch = [qps[(off + i) % len(qps)] for i in range(per_step)]
            off += per_step
            t0 = time.perf_counter()
            pool.map(_oracle_solve_one, batch, chunksize=1)
            dt = time.perf_counter() - t0
            vals.append(len(batch) / dt)
            t_all += dt
            done += len(batch)
    value = done / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_of(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} instances ({per_step} per step) solved to 1e-6 by the FP64 C "
                                   f"oracle, {cores} worker processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2602_23967_b300 import pdhcg
    pdhcg.lib()
    prm = pdhcg.default_params(precision=args.precision, eps_tol=EPS)
    stream = torch.cuda.Stream()
    qps = instances(args.count, rank, world, args.scaling)
    tune = None
    if args.autotune:
        prm, tune = pdhcg.autotune(qps[:512], prm, stream=stream.cuda_stream)
    probs = pdhcg.create_batch(qps, prm, stream=stream.cuda_stream)

    def step():
        return pdhcg.solve_batch(probs, want_solutions=False)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.time()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
            out = step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.time() - wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), world, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    value = job_throughput(world, args.count, args.steps, total_ms, args.scaling)
    iters = np.array([r["iterations"] for r in out])
    statuses = [r["status_name"] for r in out]
    kkt = np.array([max(r["r_primal"], r["r_dual"], r["r_gap"]) for r in out])

    # roofline of the batched solve kernel (algorithmic bytes / device time per launch)
    alg = sum(algorithmic_bytes(q, int(r["iterations"])) for q, r in zip(qps, out))
    launch_s = (total_ms / args.steps) * 1e-3
    peaks, peak_kind = measured_peaks()
    achieved = alg / launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic_per_launch(args.count),
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": alg,
                "note": "algorithmic bytes count every matrix/vector pass of every PDHG step; each instance "
                        "stays in shared memory / L1 inside its CTA, so measured DRAM traffic (from a "
                        "512-instance ncu capture, scaled by instance count) is far below them"}

    result = {}
    if rank == 0:
        # plain one-at-a-time solver on a sample of the same instances
        plain = probs[: args.plain_sample]
        xo = torch.empty(max(p.n for p in plain), dtype=torch.float64, device="cuda")
        yo = torch.empty(max(max(p.m for p in plain), 1), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.time()
        for p in plain:
            p.solve_dev(xo, yo)
        torch.cuda.synchronize()
        plain_sps = len(plain) / (time.time() - t0)

        # end to end through the public API: upload + setup + solve + download, from host data
        h2d = sum(input_bytes(q) for q in qps)
        d2h = sum(8 * (q.n + q.m) for q in qps) + len(qps) * 160
        e2e_t = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.time()
            ps = pdhcg.create_batch(qps, prm, stream=stream.cuda_stream)
            sol = pdhcg.solve_batch(ps, want_solutions=True)
            torch.cuda.synchronize()
            e2e_t.append(time.time() - t0)
            for p in ps:
                p.close()
        e2e_sps = args.count / float(np.median(e2e_t))

        # CPU oracle baseline on a bounded sample, and the error against it
        cpu_sps, cpu_res, cpu_dt = cpu_oracle_sample(qps, args.cpu_sample)
        objs = np.array([r["primal_obj"] for r in out[: len(cpu_res)]])
        oobj = np.array([r["primal_obj"] for r in cpu_res])
        obj_err = float(np.max(np.abs(objs - oobj) / (1 + np.abs(oobj)))) if len(cpu_res) else None
        # independent FP64 KKT of every benchmark solution (the last end-to-end solve's)
        kkt64 = [fp64_kkt(q, x, y) for q, (x, y, _) in zip(qps, sol)]
        serving = serving_leg(args, stream.cuda_stream) if args.serve_rates else None
        large = large_instance_leg(args, stream, peaks["hbm_gbs"]) if args.large_iters > 0 else None
        whole = whole_solve_leg(args, stream) if args.whole_eps else None
        result = dict(plain_sps=plain_sps, e2e_sps=e2e_sps, h2d=h2d, d2h=d2h, cpu_sps=cpu_sps,
                      cpu_n=len(cpu_res), cpu_dt=cpu_dt, obj_err=obj_err, serving=serving, large=large,
                      whole=whole, kkt64_max=float(max(kkt64)), kkt64_n=len(kkt64))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None,
            "dtype": {"mixed": "f32 matrix values, f64 vectors and reductions", "fp64": "f64",
                      "dfloat": "f32x2 (double-float) vectors on the FP32 pipe, f32 matrix values, f64 reductions",
                      "fp32": "f32 (f64 reductions)"}[args.precision],
            "data": "synthetic",
            "config": config_of(args),
            "plain_solves_per_s": result.get("plain_sps"),
            "batched_vs_plain": value / world / result["plain_sps"] if result.get("plain_sps") else None,
            "solved_optimal": statuses.count("OPTIMAL"), "instances": len(statuses),
            "kkt_max": float(kkt.max()),
            "kkt_fp64_max": result.get("kkt64_max"),
            "kkt_fp64_note": f"max over all {result.get('kkt64_n')} solutions of the relative KKT residual "
                             "(Sec. 4.2) recomputed on the host in FP64 from the problem data",
            "iterations_mean": float(iters.mean()),
            "iterations_max": int(iters.max()),
            "error_vs_fp64_oracle": {"objective_rel_max": result.get("obj_err"),
                                     "sample": result.get("cpu_n")},
            "roofline": roofline,
            "cpu_baseline": {"value": result.get("cpu_sps"), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {result.get('cpu_n')} of the {args.count} instances, full FP64 "
                                       f"oracle solves to 1e-6 ({result.get('cpu_dt', 0):.1f} s, one thread)"},
            "e2e": {"value": result.get("e2e_sps"), "unit": UNIT, "h2d_bytes_per_step": result.get("h2d"),
                    "d2h_bytes_per_step": result.get("d2h")},
            "serving": result.get("serving"),
            "large_instance_spmv": result.get("large"),
            "whole_solves": result.get("whole"),
            "autotune": tune,
            "gpu_launches": args.steps,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    for p in probs:
        p.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ablation_inner_tolerance(args):
    """Sec. 6.3's question on these synthetic inputs: outer steps, inner steps and device time
    to relative KKT 1e-6 with the adaptive inner tolerance of Sec. 3.3 against
    fixed inner tolerances (gamma = 0: eps_k = eps_min from the second step)."""
    import torch
    from paper_2602_23967_b300 import pdhcg
    torch.cuda.set_device(0)
    cases = [(f"random_qp n=200 seed {s}", W.random_qp(seed=s)) for s in range(8)]
    cases += [("large sparse n=2e5", W.large_sparse_qp(n=200_000, m=100_000, seed=0))]
    rules = {"adaptive (Sec. 3.3)": {}, "fixed 1e-9": dict(gamma_inner=0.0, eps_inner_min=1e-9),
             "fixed 1e-6": dict(gamma_inner=0.0, eps_inner_min=1e-6)}
    rows = []
    for name, qp in cases:
        for rule, kw in rules.items():
            p = pdhcg.Problem(qp, pdhcg.default_params(precision=args.precision, eps_tol=EPS,
                                                       max_iter=200_000, time_limit_s=120.0, **kw))
            try:
                _, _, r = p.solve()
            finally:
                p.close()
            rows.append({"instance": name, "rule": rule, "status": r["status_name"],
                         "outer": r["iterations"], "inner": r["inner_iterations"],
                         "seconds": r["solve_seconds"]})
    print(json.dumps({"ablation": "inner-tolerance", "precision": args.precision, "rows": rows}), flush=True)


def run_ablation_inner_solver(args):
    """Reading D1's two inner solvers for a non-diagonal Q with finite bounds:
    projected BB gradient (AUTO) against CG on the lifted problem (bounds as rows
    of A), to relative KKT 1e-6."""
    import torch
    from paper_2602_23967_b300 import pdhcg
    torch.cuda.set_device(0)
    cases = [(f"random_qp n=200 seed {s}", W.random_qp(seed=s)) for s in range(8)]
    cases += [("large sparse n=2e5", W.large_sparse_qp(n=200_000, m=100_000, seed=0))]
    rows = []
    for name, qp in cases:
        for inner in ("bb", "cg_lifted"):
            p = pdhcg.Problem(qp, pdhcg.default_params(precision=args.precision, eps_tol=EPS, inner=inner,
                                                       max_iter=200_000, time_limit_s=120.0))
            try:
                _, _, r = p.solve()
            finally:
                p.close()
            rows.append({"instance": name, "inner": inner, "status": r["status_name"],
                         "outer": r["iterations"], "inner_steps": r["inner_iterations"],
                         "seconds": r["solve_seconds"]})
    print(json.dumps({"ablation": "inner-solver", "precision": args.precision, "rows": rows}), flush=True)


def main():
    args = parse()
    if args.ablation == "inner-tolerance":
        run_ablation_inner_tolerance(args)
        return
    if args.ablation == "inner-solver":
        run_ablation_inner_solver(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
