#!/usr/bin/env python
"""GoDec-BRP benchmark: iterations/s and HBM roofline on the 10000 x 10000, r = 50,
q = 2, k = 1e6 float32 workload (synthetic, seeded).

A step is one iteration of Algorithm 1 (all passes of the L-step, the S-step
and the update of X - S).  The timed region runs K iterations from S = 0 with
X resident in HBM (X and X - S are 400 MB each, above the 129 MB L2, so no
flush is needed between iterations).  Multi-GPU runs are independent replicas
(one problem per rank, no collective on the data path): weak scaling.

--impl reference times the float64 CPU oracle on the same full-size workload: each
step is one oracle iteration of Algorithm 1 on the whole 10000 x 10000 matrix.

The default line also carries "forms": clocked timing records of the other
configurations, each against its stated comparison (the 500 x 500 case against the
oracle, the precision form against the float32 form, the batched form against the
same problems one by one, the differentiated form's backward against its forward).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GoDec-BRP iters/s & HBM GB/s at 10k×10k r=50 (vs plain FP32), rel err vs FP64"
UNIT = "iterations/s"
M = N = 10000
R, K_CARD, Q = 50, 1000000, 2
WORKLOAD = ("plain GoDec-BRP float32, X = U V^T + S + G, m = n = 10000, rank-50 N(0,1) factors, "
            "1% sparse U[-20,20], noise sigma 1e-2; r = 50, k = 1e6, q = 2, iterations from S = 0")
BASELINE_ITERS = 3        # full-size oracle iterations of the GPU arm's cpu_baseline


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the C1/C3/C4/C5 timing records")
    ap.add_argument("--kernel", choices=["product", "product_t", "iteration", "backward", "precision", "batched", "c1",
                                         "grebsmo", "naive", "lingodec", "mse", "first_projection"], default=None,
                    help="profiling aid: run one kernel family on a small case and exit (no JSON line)")
    ap.add_argument("--size", type=int, default=8192)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        under_load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(under_load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def pass_traffic():
    """DRAM bytes per launch of the streaming product (dram__bytes_read.sum +
    dram__bytes_write.sum of one ncu capture, scaled to the benchmark's size) from the
    committed summary, if it was taken on the current kernel source; else None."""
    import hashlib
    src = os.path.join(ROOT, "paper_1309_0302_gb300", "csrc", "k_tc.cu")
    p = os.path.join(ROOT, "profiles", "k_prod_tc_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = dict(line.strip().split("=", 1) for line in open(p) if "=" in line and not line.startswith("#"))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return float(kv["dram_bytes_per_launch"]) if kv.get("source_sha") == h else None


def oracle_steps(X32, A1_32, steps: int, warmup: int):
    """The float64 oracle on the full workload: `warmup` untimed then `steps` timed
    iterations of Algorithm 1 (one oracle.godec_step each, continuing the trajectory from
    S = 0).  Returns (iterations/s, per-iteration seconds, threads used)."""
    import numpy as np

    import oracle
    X, A1 = X32.astype(np.float64), A1_32.astype(np.float64)
    S_idx, S_val = np.zeros(0, np.int64), np.zeros(0)
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        st = oracle.godec_step(X, A1, S_idx, S_val, K_CARD, Q)
        if i >= warmup:
            times.append(time.perf_counter() - t0)
        S_idx, S_val = st["S_idx"], st["S_val"]
    return len(times) / sum(times), times, blas_threads()


def blas_threads() -> int:
    """Threads the oracle's BLAS runs on (numpy's OpenBLAS honours OMP/OPENBLAS env)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count()


def replica_seed(rank: int) -> int:
    """Seed of rank r's replica: every rank solves its own problem of the same shape."""
    return 1309 + rank


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time: the slowest rank's (all-reduce MAX; CUDA tensor under NCCL, CPU
    tensor under gloo).  Without a process group, the local time."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, steps: int, ms: float) -> float:
    """Whole-job iterations/s: the iterations of all ws replicas over the slowest rank's time."""
    return ws * steps / (ms / 1000.0)


def emit(line: dict):
    print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import synth
    d = synth.lowrank_sparse(M, N, R, K_CARD, -20.0, 20.0, 1e-2, replica_seed(0), "c2")
    warm = min(args.warmup, 1)
    t0 = time.perf_counter()
    rate, times, cores = oracle_steps(d["X"], d["A1"], args.steps, warm)
    wall = time.perf_counter() - t0
    emit({"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": warm, "ms_per_step": 1000.0 / rate, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": WORKLOAD, "m": M, "n": N, "r": R, "k": K_CARD, "q": Q},
          "cpu_baseline": {"kind": "oracle", "cores": cores, "value": rate, "unit": UNIT,
                           "sample": f"the whole workload: {warm} untimed and {args.steps} timed float64 "
                                     f"oracle iterations of the full {M} x {N} matrix from S = 0 "
                                     f"({wall:.1f} s wall in all)"},
          "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_gb300(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d = synth.lowrank_sparse(M, N, R, K_CARD, -20.0, 20.0, 1e-2, replica_seed(rank), "c2")
    X = torch.from_numpy(d["X"]).cuda()
    A1 = torch.from_numpy(d["A1"]).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = G.GoDec(X, A1, R, K_CARD, Q, tol=1e-7, max_iter=args.steps, stream=stream)
        g.iterate(max(1, args.warmup))          # warm-up iterations; captures the graph
        g.reset()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rel = g.iterate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        if dist:
            dist.barrier()
        info = g.info()
        # per-kernel device times of the same iterations (eager launches bracketed by events)
        g.reset()
        prof = g.profile(args.steps)
        g.close()
    value = job_value(ws, args.steps, ms)
    npass = prof["launches"]["product"]
    pass_ms = prof["ms"]["product"] / max(npass, 1)
    achieved = prof["bytes_product"] / (pass_ms / 1000.0) / 1e9
    peak, peak_src = peaks()
    passes_per_iter = npass / args.steps
    bytes_iter = iteration_bytes(M, N, R, K_CARD, Q)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "r": R, "k": K_CARD, "q": Q,
                   "iterations": args.steps, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (X and X - S are 400 MB each); no flush"},
        "rel_err": rel,
        "roofline": {"bound": "hbm", "kernel": "streaming product over X - S", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": pass_traffic(),
                     "peak_source": peak_src, "avg_launch_ms": pass_ms,
                     "bytes_per_launch": prof["bytes_product"]},
        "iteration_roofline": {"achieved": bytes_iter * (value / ws) / 1e9, "unit": "GB/s",
                               "frac": bytes_iter * (value / ws) / 1e9 / peak,
                               "bytes_per_iter": bytes_iter,
                               "bytes_rule": "algorithmic: (6q+3) passes over the 4mn-byte matrix (6q+2 "
                                             "products with X A1 cached, one S-step pass), (6q+2) reads and "
                                             "one write of the 12k-byte COO S, skinny operands in and out",
                               "product_launches_per_iter": passes_per_iter,
                               "residual_passes_per_iter": max(1, int(info["select_passes"]))},
        "kernel_ms_per_iter": {k: v / args.steps for k, v in prof["ms"].items()},
        "clocks": ck,
        "gpu_launches": int(info["launches_per_iter"]) * args.steps,
        "path": {k: info[k] for k in ("svd_sweeps", "select_passes", "exact_iters", "rank_drops", "chol_shifts")},
    }
    if not args.no_e2e:
        line["e2e"] = e2e(args, d)
    if rank == 0 and ws == 1 and not args.no_forms:
        line["forms"] = {"c1": form_c1(), "c3_precision": form_c3(), "c4_batched": form_c4(),
                         "c5_differentiated": form_c5(), "grebsmo": form_grebsmo(), "naive": form_naive(),
                         "lingodec": form_lingodec(), "mse": form_mse(), "first_projection": form_first_projection()}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, times, cores = oracle_steps(d["X"], d["A1"], BASELINE_ITERS, 0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{BASELINE_ITERS} float64 oracle iterations of the full {M} x {N} "
                                          f"workload from S = 0 ({sum(times):.1f} s)"}
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        emit(line)


def e2e(args, d):
    """Same metric through godec_run_host: pinned host X and A1 in, L factors and S out,
    all copies and allocations inside the timed call."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    Xh = torch.empty((M, N), dtype=torch.float32).pin_memory()
    Xh.numpy()[:] = d["X"]
    Ah = torch.from_numpy(d["A1"]).pin_memory()
    out = {"U": torch.empty((M, R)).pin_memory().numpy(), "V": torch.empty((N, R)).pin_memory().numpy(),
           "sigma": np.empty(R, np.float32), "S_idx": torch.empty(K_CARD, dtype=torch.int64).pin_memory().numpy(),
           "S_val": torch.empty(K_CARD, dtype=torch.float32).pin_memory().numpy()}
    G.run_host(Xh.numpy(), Ah.numpy(), R, K_CARD, Q, 1, out=out)          # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.run_host(Xh.numpy(), Ah.numpy(), R, K_CARD, Q, args.steps, out=out)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = 4.0 * M * N + 4.0 * N * R
    d2h = 4.0 * (M + N) * R + 4.0 * R + 12.0 * K_CARD
    return {"value": args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
            "d2h_bytes_per_step": d2h / args.steps,
            "note": "one godec_run_host call per measurement: H2D of X and A1, K iterations, D2H of L "
                    "factors and sorted S; bytes per step = bytes per call / K"}


def iteration_bytes(m, n, r, k, q) -> float:
    """Algorithmic bytes of one iteration of Algorithm 1 in the streaming design: 6q+3 passes
    over the 4mn-byte matrix (6q+2 chain products once X A1 is cached, plus one S-step pass),
    6q+2 reads and one write of the 12-byte-per-entry COO S, and the skinny operands read and
    written by each of the 6q+3 products."""
    P = 6 * q + 3
    return P * 4.0 * m * n + (P - 1) * 12.0 * k + 12.0 * k + P * 2 * 4.0 * (m + n) * r


def _timed(stream, f, reps: int):
    """Milliseconds per call of f over reps calls, CUDA events on `stream`, with nvidia-smi
    clock samples over the same region."""
    import torch
    ck = Clocks(torch.cuda.current_device())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ck.start()
    ev[0].record(stream)
    for _ in range(reps):
        f()
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps, ck.stop()


def form_c1():
    """C1 (500 x 500, rank 10, k = 12500, q = 1; L2-resident, so iterations/s only): GPU
    iterations (graph replays) against the float64 oracle on all host cores and on one, and a
    solve to tol 1e-7."""
    import torch

    import oracle as O
    import paper_1309_0302_gb300 as G
    import synth
    d = synth.config_c1()
    X, A1 = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["A1"]).cuda()
    st = torch.cuda.current_stream()
    g = G.GoDec(X, A1, d["r"], d["k"], d["q"], tol=-1.0, max_iter=1 << 30)
    g.iterate(3)
    ms, ck = _timed(st, lambda: g.iterate(200), 10)
    ms /= 200
    g.close()
    g = G.GoDec(X, A1, d["r"], d["k"], d["q"], tol=1e-7, max_iter=50)
    t0 = time.perf_counter()
    it, rel = g.solve()
    t_solve = time.perf_counter() - t0
    g.close()
    t0 = time.perf_counter()
    O.godec(d["X"], d["A1"], d["k"], d["q"], tol=-1.0, max_iter=10)
    o_all = (time.perf_counter() - t0) / 10
    code = ("import sys, time; sys.path.insert(0, %r); import synth, oracle as O; d = synth.config_c1(); "
            "t0 = time.perf_counter(); O.godec(d['X'], d['A1'], d['k'], d['q'], tol=-1.0, max_iter=10); "
            "print((time.perf_counter() - t0) / 10)") % ROOT
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    o_one = float(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                 check=True).stdout.strip().splitlines()[-1])
    return {"workload": "500 x 500, rank 10, k = 12500 U[-10,10], sigma 1e-3; r = 10, q = 1",
            "gpu_iterations_per_s": 1e3 / ms, "gpu_ms_per_iter": ms, "gpu_timed_iterations": 2000,
            "solve_tol_1e-7": {"iterations": it, "rel_err": rel, "wall_ms": t_solve * 1e3},
            "oracle_iterations_per_s": {"all_cores": 1.0 / o_all, "cores": blas_threads(), "one_core": 1.0 / o_one},
            "note": "L2-resident (1 MB matrix): no HBM roofline", "clocks": ck}


def form_c3():
    """C3 (76800 x 1000, r = 3, k = 1.2e6, q = 2): the precision form (float16 chain +
    float32 correction) against the plain float32 form on the same input, 100 timed
    iterations each after 2 warm-up ones; the two L's distance afterwards."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    d = synth.config_c3()
    X, A1 = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["A1"]).cuda()
    st = torch.cuda.current_stream()
    out, Ls = {}, {}
    for name, prec in (("float32", G.PREC_FP32), ("precision", G.PREC_BF16_REFINE)):
        g = G.GoDec(X, A1, d["r"], d["k"], d["q"], tol=-1.0, max_iter=1 << 30, precision=prec)
        g.iterate(2)
        ms, ck = _timed(st, lambda: g.iterate(20), 5)
        ms /= 20
        out[name] = {"ms_per_iter": ms, "iterations_per_s": 1e3 / ms, "clocks": ck,
                     "exact_path_iterations": g.info()["exact_iters"]}
        Ls[name] = [t.double().cpu().numpy() for t in g.L()]
        g.close()
    (Ua, sa, Va), (Ub, sb, Vb) = Ls["float32"], Ls["precision"]
    Aa, Ab = Ua * sa, Ub * sb
    aa, bb, ab = (np.sum((P.T @ Q) * (R_.T @ S_)) for P, Q, R_, S_ in
                  ((Aa, Aa, Va, Va), (Ab, Ab, Vb, Vb), (Aa, Ab, Va, Vb)))
    m, n = d["X"].shape
    return {"workload": "76800 x 1000 video-shaped synthetic, r = 3, k = 1.2e6, q = 2",
            "float32": out["float32"], "precision": out["precision"],
            "speedup_precision_over_float32": out["float32"]["ms_per_iter"] / out["precision"]["ms_per_iter"],
            "L_distance_after_102_iterations": float(np.sqrt(max(aa + bb - 2 * ab, 0.0)) / np.sqrt(aa)),
            "algorithmic_bytes_per_iter": {"precision": 14 * 2.0 * m * n + 2 * 4.0 * m * n,
                                           "float32": 15 * 4.0 * m * n}}


def form_c4():
    """C4 (64 problems, m, n log-uniform in [256, 4096], r in 2..32, q = 1): the tuned batch
    (one graph launch per batch iteration) against the same problems one by one."""
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    ds = synth.config_c4()
    Xs = [torch.from_numpy(d["X"]).cuda() for d in ds]
    A1s = [torch.from_numpy(d["A1"]).cuda() for d in ds]
    rs, ks, qs = [d["r"] for d in ds], [d["k"] for d in ds], [d["q"] for d in ds]
    nbytes = sum(iteration_bytes(*d["X"].shape, d["r"], d["k"], d["q"]) for d in ds)
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    b = G.GoDecBatch(Xs, A1s, rs, ks, qs, tune=True)
    t_init = time.perf_counter() - t0
    b.iterate(2)
    ms_b, ck_b = _timed(st, lambda: b.iterate(20), 10)
    ms_b /= 20
    tun = b.tuning()
    paths = [b.problem(j).info() for j in range(len(ds))]
    b.close()
    single = 0.0
    cks = []
    for j in range(len(ds)):
        g = G.GoDec(Xs[j], A1s[j], rs[j], ks[j], qs[j], tol=-1.0, max_iter=1 << 30)
        g.iterate(2)
        ms, ck = _timed(st, lambda: g.iterate(20), 1)
        single += ms / 20
        cks.append(ck)
        g.close()
    ck_single = {"sm_mhz": statistics.median([c["sm_mhz"] for c in cks if c.get("sm_mhz")] or [0]),
                 "sm_max_mhz": max([c["sm_max_mhz"] or 0 for c in cks]),
                 "reasons": sorted({r_ for c in cks for r_ in c["reasons"]})}
    return {"workload": "64 problems, m, n log-uniform in [256, 4096], r in 2..32, 2-5 % sparse, q = 1",
            "batch": {"ms_per_batch_iter": ms_b, "problem_iterations_per_s": 64e3 / ms_b,
                      "algorithmic_GBps": nbytes / ms_b / 1e6, "policy": tun["policy"],
                      "policy_ms": tun["policy_ms"], "init_s_with_tuning": t_init, "clocks": ck_b,
                      "exact_path_iterations": sum(p_["exact_iters"] for p_ in paths),
                      "iterations": sum(p_["iter"] for p_ in paths), "alarms": sum(p_["alarms"] for p_ in paths)},
            "one_by_one": {"ms_per_round_of_64": single, "problem_iterations_per_s": 64e3 / single,
                           "clocks": ck_single},
            "speedup_batch_over_one_by_one": single / ms_b}


def form_c5():
    """C5 (4096 x 4096, r = 20, q = 0, T = 10): the differentiated form's backward
    (godec_backward) against its forward (T iterations, context set-up included)."""
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    d = synth.config_c5()
    r, k, T = d["r"], d["k"], d["T"]
    X, A1 = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["A1"]).cuda()
    st = torch.cuda.current_stream()
    box = {}

    def forward():
        g = G.GoDec(X, A1, r, k, 0, tol=0.0, max_iter=T)
        sup = []
        for t in range(T):
            g.iterate(1)
            if t < T - 1:
                sup.append(g.S()[0].clone())
        box["L"] = g.L()
        box["sup"] = sup
        g.close()

    forward()
    ms_f, ck_f = _timed(st, forward, 10)
    U, s, V = box["L"]
    gU = torch.cat([2.0 * U * s, -2.0 * torch.from_numpy(d["Ustar"]).float().cuda()], 1).contiguous()
    gV = torch.cat([V, torch.from_numpy(d["Vstar"]).float().cuda()], 1).contiguous()
    G.backward(X, A1, T, box["sup"], gU=gU, gV=gV)
    ms_b, ck_b = _timed(st, lambda: G.backward(X, A1, T, box["sup"], gU=gU, gV=gV), 40)
    m, n = d["X"].shape
    return {"workload": "4096 x 4096, rank 20, 2 % sparse, r = 20, q = 0, T = 10, loss ||L_T - L*||^2",
            "forward_ms": ms_f, "backward_ms": ms_b, "backward_over_forward": ms_b / ms_f,
            "forward_algorithmic_bytes": T * 3 * 4.0 * m * n, "clocks_forward": ck_f, "clocks_backward": ck_b}


def form_grebsmo():
    """GreBsmo (Sec. 3.2.1) on the video-shaped 76800 x 1000 matrix of the precision-form
    workload: rank increments of 1 up to 3, 10 inner steps per stage, lambda = 0.15 (the blob
    foreground goes to S); time to the stop, per inner step."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    d = synth.config_c3()
    X = torch.from_numpy(d["X"]).cuda()
    m, n = d["X"].shape
    om = torch.from_numpy(synth.gaussian(1309, "bench/greb/omega", (3, n, 7)).astype(np.float32)).cuda()
    st = torch.cuda.current_stream()
    box = {}

    def run():
        g = G.GreBsmo(X, om, 0.15, 1, 10, 0.0, 3, oversample=6, q_inc=4, s_cap=16_000_000)
        box["r"], box["errs"] = g.run()
        box["iter"] = g.info()["iter"]
        box["nnz"] = g.info()["nnz"]
        g.close()

    run()
    ms, ck = _timed(st, run, 3)
    return {"workload": "76800 x 1000 video-shaped synthetic, lambda 0.15, dr 1, K 10, r_max 3, "
                        "random-projection increments (6 extra columns, 4 power steps)",
            "ms_to_stop_incl_context": ms, "inner_steps": box["iter"], "ms_per_inner_step": ms / box["iter"],
            "rank": box["r"], "stage_errors": box["errs"], "support_of_S": box["nnz"], "clocks": ck}


def form_naive():
    """Naive GoDec (eq. raw_lss, truncated-SVD L-step) at the 10000 x 10000, r = 50 workload,
    2 power steps per L-step: iterations/s beside the BRP form's."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    d = synth.lowrank_sparse(M, N, R, K_CARD, -20.0, 20.0, 1e-2, replica_seed(0), "c2")
    X = torch.from_numpy(d["X"]).cuda()
    p = G.naive_columns(M, N, R)
    om = torch.from_numpy(synth.gaussian(1309, "bench/naive/omega", (N, p)).astype(np.float32)).cuda()
    st = torch.cuda.current_stream()
    g = G.NaiveGoDec(X, om, R, K_CARD, q=2, tol=-1.0, max_iter=1 << 30)
    g.iterate(3)
    ms, ck = _timed(st, lambda: g.iterate(10), 3)
    ms /= 10
    rel = g.info()["rel_err"]
    g.close()
    return {"workload": "10000 x 10000, rank 50, 1 % sparse, r = 50, subspace iteration over 58 columns, "
                        "2 power steps per L-step", "ms_per_iter": ms, "iterations_per_s": 1e3 / ms,
            "rel_err_after_16_iterations": rel, "clocks": ck}


def form_first_projection():
    """The chain's first projection (X - S) A1 both ways on the 10000 x 10000, r = 50, q = 2
    shape with a sparser S (k = 10^5, 0.1 %): streamed over Z like the other products
    (GODEC_FLAG_DENSE_FIRST, the default), or X A1 - S A1 from the cached X A1
    (GODEC_FLAG_SPARSE_FIRST).  Whole iterations, CUDA events, same input; the counts of
    alarms and exact-path iterations say how many of the timed iterations were redone."""
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    k = 100000
    d = synth.lowrank_sparse(M, N, R, k, -20.0, 20.0, 1e-2, replica_seed(0), "c2_sparse")
    X, A1 = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["A1"]).cuda()
    st = torch.cuda.current_stream()
    out = {}
    for name, flags in (("sparse", G.FLAG_SPARSE_FIRST), ("dense", G.FLAG_DENSE_FIRST)):
        g = G.GoDec(X, A1, R, k, Q, tol=-1.0, max_iter=1 << 30, flags=flags)
        g.iterate(6)
        ms, ck = _timed(st, lambda: g.iterate(10), 3)
        ms /= 10
        info = g.info()
        out[name] = {"ms_per_iter": ms, "iterations_per_s": 1e3 / ms, "rel_err": info["rel_err"],
                     "alarms": info["alarms"], "exact_path_iterations": info["exact_iters"],
                     "iterations": info["iter"], "clocks": ck}
        g.close()
    return {"workload": "10000 x 10000, rank 50, k = 1e5 (0.1 %) U[-20, 20], noise 1e-2; r = 50, q = 2",
            "sparse_first": out["sparse"], "dense_first": out["dense"],
            "speedup_sparse_over_dense": out["dense"]["ms_per_iter"] / out["sparse"]["ms_per_iter"]}


def form_lingodec():
    """LinGoDec (Sec. 4.3) on the paper's synthetic recipe at 20000 users x 5000 items,
    d = 50 item features, rank 10, 5 % +-1 outliers: iterations/s."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    m, n, dd, r = 20000, 5000, 50, 10
    W = synth.gaussian(1309, "bench/lingo/Wa", (m, r)) @ synth.gaussian(1309, "bench/lingo/Wb", (r, dd))
    F = synth.gaussian(1309, "bench/lingo/F", (n, dd))
    X = W @ F.T
    pos = synth.sample_positions(1309, "bench/lingo/S", m * n, int(0.05 * m * n))
    sg = np.where(synth.uniform(1309, "bench/lingo/sg", (pos.size,), 0.0, 1.0) < 0.5, -1.0, 1.0)
    X.ravel()[pos] += sg
    X += 1e-3 * synth.gaussian(1309, "bench/lingo/G", (m, n))
    Xg = torch.from_numpy(X.astype(np.float32)).cuda()
    Fg = torch.from_numpy(F.astype(np.float32)).cuda()
    st = torch.cuda.current_stream()
    g = G.LinGoDec(Xg, Fg, r, 0.25, s_cap=int(0.06 * m * n))
    g.iterate(2)
    ms, ck = _timed(st, lambda: g.iterate(10), 2)
    ms /= 10
    rel = g.info()["rel_err"]
    g.close()
    return {"workload": "20000 x 5000, d = 50, rank 10, 5 % +-1 outliers, lambda 0.25", "ms_per_iter": ms,
            "iterations_per_s": 1e3 / ms, "rel_err": rel, "clocks": ck}


def form_mse():
    """MSE training (Algorithm 4) on synthetic multi-label data: 20000 samples x 2000
    features, 8 labels (each sample carries each with probability 0.35), rank 5 per label,
    K = 0.5 % outliers; time per outer iteration."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    n, p, k, r = 20000, 2000, 8, 5
    Y = (synth.uniform(1309, "bench/mse/labels", (n, k), 0.0, 1.0) < 0.35).astype(np.int32)
    Y[Y.sum(axis=1) == 0, 0] = 1
    X = np.zeros((n, p))
    for i in range(k):
        B = np.linalg.qr(synth.gaussian(1309, f"bench/mse/basis{i}", (p, r)))[0].T
        rows = np.flatnonzero(Y[:, i])
        X[rows] += synth.gaussian(1309, f"bench/mse/coef{i}", (rows.size, r)) @ B * 3.0
    K = int(0.005 * n * p)
    pos = synth.sample_positions(1309, "bench/mse/out", n * p, K)
    X.ravel()[pos] += synth.uniform(1309, "bench/mse/mag", (K,), 5.0, 10.0)
    X += 1e-3 * synth.gaussian(1309, "bench/mse/noise", (n, p))
    Xg = torch.from_numpy(X.astype(np.float32)).cuda()
    iters = 4
    A1s = torch.from_numpy(synth.gaussian(1309, "bench/mse/A1", (iters, k, p, r)).astype(np.float32)).cuda()
    st = torch.cuda.current_stream()
    G.mse_train(Xg, Y, [r] * k, K, 1, A1s[:1])
    box = {}
    ms, ck = _timed(st, lambda: box.update(out=G.mse_train(Xg, Y, [r] * k, K, iters, A1s)), 1)
    return {"workload": "20000 x 2000, 8 labels, rank 5 each, 0.5 % outliers, q = 0 BRP blocks",
            "ms_per_outer_iteration_incl_setup": ms / iters, "outer_iterations": iters,
            "objective_history": box["out"]["history"], "clocks": ck}


def run_kernel_case(args):
    """Small cases for ncu captures: the streaming product on a size x size matrix
    (above the L2 size for size >= 6000), or two full iterations at size x size, r = 50."""
    import numpy as np
    import torch

    import paper_1309_0302_gb300 as G
    import synth
    n = args.size
    if args.kernel in ("product", "product_t"):
        g = np.random.default_rng(5)
        Z = torch.from_numpy(g.standard_normal((n, n)).astype(np.float32)).cuda()
        B = torch.from_numpy(g.standard_normal((n, R)).astype(np.float32)).cuda()
        f = G.mul_ZB if args.kernel == "product" else G.mul_ZtC
        for _ in range(3):
            f(Z, B)
    elif args.kernel in ("backward", "precision", "batched", "c1", "grebsmo", "naive", "lingodec", "mse",
                         "first_projection"):
        f = {"backward": form_c5, "precision": form_c3, "batched": form_c4, "c1": form_c1, "grebsmo": form_grebsmo,
             "naive": form_naive, "lingodec": form_lingodec, "mse": form_mse,
             "first_projection": form_first_projection}[args.kernel]
        print(json.dumps(f(), indent=1))
    else:
        d = synth.small_case(n, n, R, 0.01, R, Q, tag="kernel_case")
        run = G.GoDec(torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["A1"]).cuda(), R, d["k"], Q)
        run.iterate(2)
        run.close()
    torch.cuda.synchronize()
    print(f"kernel case {args.kernel} size {n}: done")


def main():
    args = parse()
    if args.kernel:
        run_kernel_case(args)
        return
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_gb300(args, ws, rank, local)


if __name__ == "__main__":
    main()
