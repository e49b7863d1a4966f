"""Benchmark: time to relative KKT 1e-5 per solve on the n = 2000 sparse-Theta
workload (m = 1000 Gaussian samples, lambda = 0.1, FP64 S), one step = one
complete solve from the FP64 covariance S (ML-cycles of the proximal-Newton
relaxation until rel. KKT <= 1e-5).  S is formed once on the GPU from the
samples before timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...    (the FP64 CPU oracle, same metric)

Prints one JSON line (rank 0).  `value` is whole-job solves/s with S already
resident in HBM; `e2e` is the same metric through the public API with pinned
host buffers (S copied in, A copied out, inside the timed region).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. KKT 1e-5 per solve (mixed vs FP64 GPU); solves/sec, p50/p99 latency"
CONFIG_ID = 2
WORKLOAD = "sparse-Theta n=2000 m=1000 lambda=0.1, fp64 S given, to rel. KKT 1e-5"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def sustained_bf16(default):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("bf16_tflops_sustained", default)
    return 1700.0


def fp64_peak_tflops(bf16_tflops):
    # FP64 contraction peak: the bf16 peak times the nominal FP64/bf16 ratio (1.25 / 2250)
    return bf16_tflops * 1.25 / 2250.0


def tf32_peak_tflops(bf16_tflops):
    # TF32 tensor peak: the measured bf16 peak times the nominal TF32/bf16 ratio (1.1 / 2.25)
    return bf16_tflops * 1.1 / 2.25


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: bench_clocks/ beside this file)
        out = os.environ.get("BENCH_CLOCKS_DIR", os.path.join(ROOT, "bench_clocks"))
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_value(local_ms, steps, world, device):
    """Whole-job throughput of `steps` solves on each of `world` ranks: the
    timed region is the slowest rank's (max over ranks), value = solves of all
    ranks / that time.  Returns (max_ms, solves_per_s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, world * steps / (max_ms * 1e-3)


def batched_job_value(local_s, local_solves, world, device):
    """Whole-job throughput of independent shards: the timed region is the
    slowest rank's, the solves are summed over ranks.  Returns (max_s,
    total_solves, solves_per_s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
    c = torch.tensor([float(local_solves)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    max_s, total = float(t.item()), int(c.item())
    return max_s, total, total / max_s


def host_cpu():
    """Logical CPUs of this host and its CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    return os.cpu_count() or 1, model or "unknown"


def oracle_solve_timed(S, lam, tol):
    """One whole FP64 oracle solve of the workload (S given) on one core:
    returns (seconds, info)."""
    import oracle

    t0 = time.perf_counter()
    _, _, info, _ = oracle.solve(S, lam, tol=tol)
    return time.perf_counter() - t0, info


_POOL_S = None


def _pool_init(S):
    global _POOL_S
    _POOL_S = S


def _pool_solve(args):
    lam, tol = args
    t, info = oracle_solve_timed(_POOL_S, lam, tol)
    return t, info["relaxations"], info["status"], info["rel_kkt"]


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, variant=None):
    """DRAM bytes per launch of the dominant class from a committed ncu summary
    (the entry "class:variant" when there is one, e.g. the inner solver of
    cd_sweeps), or None when the summary is missing or was taken on other
    kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(f"{kernel_class}:{variant}") if variant else None
    e = e or d.get(kernel_class)
    if not e or e.get("source_hash") != source_hash(e.get("sources", [])):
        return None
    return e.get("dram_bytes_per_launch")


def run_reference(args):
    """The oracle arm: every step is one whole FP64 oracle solve of the
    workload (the same S, lambda and tolerance), run as it stands, one solve
    per process on the host's cores (spawned workers, at most one per core).
    value = timed solves / wall time of the timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp

    from paper_1607_00315_gb300 import synth
    import oracle

    oracle.build()
    p = synth.config_problem(CONFIG_ID)
    S = oracle.form_S(p.X)
    ncpu, model = host_cpu()
    workers = max(1, min(ncpu, args.steps, 16))
    with mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(S,)) as pool:
        if args.warmup > 0:
            pool.map(_pool_solve, [(p.lam, p.tol)] * args.warmup, chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_pool_solve, [(p.lam, p.tol)] * args.steps, chunksize=1)
        wall = time.perf_counter() - t0
    per = [r[0] for r in res]
    value = args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": p.n, "m": p.m, "lambda": p.lam, "tol": p.tol,
                   "input": "S (fp64) given"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": workers, "kind": "oracle",
                         "host_cpus": ncpu, "cpu_model": model,
                         "sample": f"whole oracle solves of the workload to rel. KKT {p.tol}, one per "
                                   f"process on {workers} of {ncpu} host CPUs ({model}); "
                                   f"{args.steps} timed after {args.warmup} warm-up; single solve "
                                   f"{np.mean(per):.2f} s mean, {res[0][1]} relaxations, "
                                   f"rel. KKT {res[0][3]:.2e}"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _gen_serving(row):
    from paper_1607_00315_gb300 import synth

    _, n, lam, seed = row
    return synth.serving_problem(n, lam, seed).X


def run_batched(args):
    """Lambda paths of many small independent instances (n ~ U[32, 512], m = 2n,
    tridiagonal / sparse generators alternating), each path warm started.
    Engine "fused" (default): one glasso_solve_batch_fused call, every solve in
    one persistent launch (a CTA per path, FP64, all control on the device);
    engine "slots": one glasso_solve_batch call, paths run concurrently
    through the host-driven serving slots (mixed precision).  Under torchrun
    the instances are split over the ranks (shard.balanced_partition) and each
    rank solves its share; the time is the slowest rank's.  value = solves/s
    over all instances x 4 lambdas (latency: each solve's own time)."""
    import torch
    import torch.distributed as dist

    from paper_1607_00315_gb300 import build, glasso, shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    # every instance with its lambda path is one unit; units are split over
    # the ranks by the greedy cost balance (no collective on the data path)
    allp = synth.batch_problems(args.instances)
    parts = shard.balanced_partition([shard.unit_cost(p.n, len(synth.LAMBDA_PATH)) for p in allp],
                                     world)
    probs = [allp[k] for k in parts[rank]]
    fused = args.batch_engine == "fused"
    ctx = glasso.Context(local, precision=glasso.MIXED)
    inner = "cd" if fused else args.batch_inner
    run = ctx.solve_batch_fused if fused else ctx.solve_batch

    def make(ps):
        plist, outs = [], []
        for p in ps:
            for lam in synth.LAMBDA_PATH:
                plist.append(glasso.Context.problem(p.X, lam, 1e-5, samples=True,
                                                    screen=args.screen and not fused, inner=inner))
                outs.append(np.empty((p.n, p.n)))
        return plist, outs

    wp, wo = make(probs[:16])
    run(wp, wo, warm_from_prev=True)  # warm-up
    plist, outs = make(probs)
    if fused:
        ctx.set_profiling(True)  # the fused kernel's own per-step clocks (no events)
        ctx.get_profile(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s, infos = run(plist, outs, warm_from_prev=True)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    share = None
    if fused:
        prof = ctx.get_profile()
        names = ("factorisations", "inverses", "scans_and_hierarchy", "cd_sweeps", "line_searches")
        cls = [prof[glasso.PROF_NAMES[c]]["ms"] for c in range(len(names))]
        tot = sum(cls)
        share = {nm: (v / tot if tot > 0 else 0.0) for nm, v in zip(names, cls)}
    ctx.close()
    max_s, total, value = batched_job_value(dt, len(plist), world, dev)
    lat = [i["seconds"] * 1e3 for i in infos]
    nfail = sum(1 for i in infos if i["status"] != 0)
    fl = sum(i["flops"] for i in infos)
    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, (lat, nfail, int(s), fl))
        lat = [x for g in gathered for x in g[0]]
        nfail = sum(g[1] for g in gathered)
        s = next((g[2] for g in gathered if g[2] != 0), 0)
        fl = sum(g[3] for g in gathered)
        dist.destroy_process_group()
    if rank != 0:
        return 0
    per = np.array(lat)
    line = {
        "metric": "batched lambda paths: solves/sec, per-solve latency p50/p99",
        "value": value, "unit": "solves/s", "n_gpus": world, "higher_is_better": True,
        "scaling": "strong",  # the instance set is fixed; more ranks split it
        "dtype": "f64" if fused else "mixed(f32/tf32+f64)", "data": "synthetic", "status": int(s),
        "config": {"workload": f"{args.instances} instances, n ~ U[32, 512], m = 2n, "
                               f"tridiagonal/sparse alternating, lambda path {list(synth.LAMBDA_PATH)} "
                               f"warm started, tol 1e-5, samples X (fp64) on the host",
                   "engine": "one persistent launch (glasso_solve_batch_fused)" if fused
                             else "host serving slots (glasso_solve_batch)",
                   "screen": bool(args.screen) and not fused, "inner": inner, "solves": total, "wall_s": max_s,
                   "parallelism": f"instances split over {world} ranks (greedy cost balance)"},
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                       "mean": float(per.mean())},
        "failed": int(nfail),
    }
    if fused:
        # the fused kernel is bound by FP64 arithmetic (its dense steps); the
        # pool measures no FP64 rate, so the peak is the nominal 1.25 TFLOP/s
        ach = fl / max_s / 1e12
        line["roofline"] = {"bound": "alu", "achieved": ach, "peak": 1.25 * world, "unit": "TFLOP/s",
                            "frac": ach / (1.25 * world), "traffic": None,
                            "peak_source": "nominal FP64 rate (no measured FP64 peak); achieved = the "
                                           "solves' algorithmic FP64 operations / the call's wall time",
                            "kernel": "k_fused_paths"}
        line["time_share"] = share  # of the CTAs' summed device time, by step
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """A Poisson request stream (n log-uniform in [64, 4096], m = n, lambda ~
    U[0.05, 0.3], sparse generator) replayed at its arrival times through
    glasso_submit / glasso_poll under a 40 GB device-memory budget; latency =
    completion - arrival (host clock).  Under torchrun every rank computes the
    same routing of the trace (shard.route_stream) and serves its own requests
    at their arrival times on its GPU; the ranks share only the start barrier
    and the final gathering of latencies."""
    import multiprocessing as mp
    import threading

    from paper_1607_00315_gb300 import shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    trace = synth.serving_trace(args.requests, rate_per_s=args.rate)
    owner = shard.route_stream([shard.unit_cost(r[1]) for r in trace], world)
    rows = [r for r, o in zip(trace, owner) if o == rank]
    # inputs generated before any CUDA work (spawned workers)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        xs = pool.map(_gen_serving, rows)
    import torch
    import torch.distributed as dist

    from paper_1607_00315_gb300 import build, glasso

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    torch.cuda.init()
    ctx = glasso.Context(local, precision=glasso.MIXED, mem_budget_bytes=40 << 30)
    # warm-up: a few requests of the trace's sizes (outputs must outlive the poll)
    wouts = [np.empty((rows[k][1], rows[k][1])) for k in range(min(8, len(rows)))]
    wt = [ctx.submit(glasso.Context.problem(xs[k], rows[k][2], 1e-5, samples=True, inner=args.batch_inner),
                     wouts[k])
          for k in range(len(wouts))]
    for t in wt:
        while ctx.poll(t, 100000)[0] == glasso.EAGAIN:
            pass
    outs = [np.empty((r[1], r[1])) for r in rows]
    done_t = [None] * len(rows)
    status = [None] * len(rows)
    tickets = [None] * len(rows)
    lock = threading.Lock()
    submitted = threading.Event()

    def collector():
        pending = set()
        while True:
            with lock:
                for k in range(len(rows)):
                    if tickets[k] is not None and done_t[k] is None and k not in pending:
                        pending.add(k)
            if not pending and submitted.is_set():
                return
            for k in list(pending):
                s, _ = ctx.poll(tickets[k], 200)
                if s != glasso.EAGAIN:
                    done_t[k] = time.perf_counter()
                    status[k] = s
                    pending.discard(k)

    th = threading.Thread(target=collector)
    if world > 1:
        dist.barrier()
    th.start()
    t0 = time.perf_counter()
    for k, (arr, n, lam, _) in enumerate(rows):
        while time.perf_counter() - t0 < arr:
            time.sleep(0.0002)
        prob = glasso.Context.problem(xs[k], lam, 1e-5, samples=True, inner=args.batch_inner)
        t = ctx.submit(prob, outs[k])
        with lock:
            tickets[k] = t
    submitted.set()
    th.join()
    ctx.close()
    arrival = np.array([r[0] for r in rows])
    done = np.array([d - t0 for d in done_t])  # seconds after this rank's start barrier
    lat = (done - arrival) * 1e3
    st_codes = [int(x) for x in status]
    first, last = (float(arrival.min()), float(done.max())) if rows else (float("inf"), 0.0)
    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, (lat.tolist(), st_codes, first, last))
        lat = np.array([x for g in gathered for x in g[0]])
        st_codes = [x for g in gathered for x in g[1]]
        first = min(g[2] for g in gathered)
        last = max(g[3] for g in gathered)
        dist.destroy_process_group()
    if rank != 0:
        return 0
    span = last - first
    line = {
        "metric": "serving stream: solves/sec (mixed), latency p50/p99",
        "value": len(trace) / span, "unit": "solves/s", "n_gpus": world, "higher_is_better": True,
        "dtype": "mixed(f32/tf32+f64)", "data": "synthetic",
        "scaling": "strong",  # the trace is fixed; more ranks split it
        "config": {"workload": f"{len(trace)} Poisson arrivals at {args.rate}/s, n log-uniform in "
                               f"[64, 4096], m = n, lambda ~ U[0.05, 0.3], sparse generator, tol 1e-5, "
                               f"samples X (fp64) on the host, 40 GB device budget",
                   "slots": int(os.environ.get("GLASSO_SERVE_SLOTS", "4")), "inner": args.batch_inner,
                   "span_s": span,
                   "parallelism": f"requests routed over {world} ranks (least modelled work)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "failed": int(sum(1 for x in st_codes if x != glasso.OK)),
    }
    print(json.dumps(line), flush=True)
    return 0


def extra_workloads(args, local, dev):
    """The other workloads, each measured once after the headline (N = 1): the
    n = 10000 solve from FP32 samples on the device (S formed on the tensor
    cores inside the solve), the batched lambda paths and the serving stream
    (each in its own bench.py process, as `--workload batched` / `serving`)."""
    import torch

    from paper_1607_00315_gb300 import glasso, synth

    out = {}
    p3 = synth.config_problem(3)
    X3 = torch.from_numpy(p3.X.astype(np.float32)).to(dev)
    with glasso.Context(local, precision=glasso.MIXED) as c3:
        stream = torch.cuda.current_stream(dev)
        c3.set_stream(stream.cuda_stream)
        A3 = torch.empty((p3.n, p3.n), dtype=torch.float64, device=dev)
        res3 = {}
        for inner in (args.inner, "pcd_cg" if args.inner == "cd" else "cd"):
            info3 = c3.solve(X3, p3.lam, tol=p3.tol, samples=True, A_out=A3, inner=inner)[2]  # warm-up
            lat3 = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info3 = c3.solve(X3, p3.lam, tol=p3.tol, samples=True, A_out=A3, inner=inner)[2]
                e1.record(stream)
                torch.cuda.synchronize()
                lat3.append(e0.elapsed_time(e1))
            ms3 = float(np.mean(lat3))
            res3[inner] = {"ms_per_solve": ms3, "solves_per_s": 1e3 / ms3, "status": info3["status"],
                           "relaxations": info3["relaxations"], "inner_iters": info3["inner_iters"],
                           "rel_kkt": info3["rel_kkt"], "nnz": info3["nnz"]}
    del X3, A3
    out["n10000_fp32_samples"] = dict(
        workload="sparse-Theta n=10000, X fp32 5000 x n on the device, S on the tensor cores "
                 "inside the solve, lambda=0.08, mixed, to rel. KKT 1e-5",
        inputs_larger_than_l2=True, **res3[args.inner], inner=args.inner,
        other_inner={k: v for k, v in res3.items() if k != args.inner})
    for name, extra in (("batched", []), ("serving", ["--requests", str(args.requests)])):
        try:
            r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", name,
                                "--batch-inner", args.batch_inner] + extra,
                               capture_output=True, text=True, timeout=600)
            line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
            out[name] = {k: line[k] for k in ("metric", "value", "unit", "latency_ms", "failed", "config",
                                              "roofline", "dtype", "time_share") if k in line}
        except Exception as e:  # reported, not fatal: the headline stands on its own
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


def run_scan(args):
    """The level-0 free-set scan alone (glasso_free_set over all pairs: the
    free set of eq. active_set, the KKT residual, tr(SA), ||A||_1) at size n
    on an iterate-like state: A = the generator's sparse precision matrix,
    W = A^-1, S the covariance of n/2 samples.  value = algorithmic GB/s:
    the upper triangles of S, W and A read once, 3 n(n+1)/2 x 8 bytes."""
    import torch

    from paper_1607_00315_gb300 import build, glasso, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    n, lam = args.scan_n, 0.1
    rng = np.random.default_rng(7000 + n)
    theta = synth.sparse_theta(n, rng)
    X = synth.gaussian_samples(theta, max(n // 2, 2), rng)
    ctx = glasso.Context(local)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    S = torch.empty((n, n), dtype=torch.float64, device=dev)
    ctx.form_S(torch.from_numpy(X).to(dev), S)
    A = torch.from_numpy(theta).to(dev)
    Wh = np.linalg.inv(theta)
    W = torch.from_numpy((Wh + Wh.T) / 2).to(dev)
    cap = n * (n + 1) // 2
    oi = torch.empty(cap, dtype=torch.int32, device=dev)
    oj = torch.empty_like(oi)
    ab = torch.empty(cap, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        cnt, rk, _ = ctx.free_set(S, W, A, lam, oi, oj, ab)
    lat = []
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cnt, rk, _ = ctx.free_set(S, W, A, lam, oi, oj, ab)
            e1.record(stream)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
    if args.profile_range:
        torch.cuda.profiler.stop()
    ms = float(np.mean(lat))
    hbm, _, src = peaks()
    gbs = 3.0 * n * (n + 1) / 2 * 8 / (ms * 1e-3) / 1e9
    line = {"metric": "level-0 free-set scan with KKT residual (glasso_free_set, all pairs)",
            "value": gbs, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"free-set scan n={n} lambda={lam}", "n": n, "free_pairs": cnt,
                       "rel_kkt": rk, "l2": "flushed between timed calls (512 MB write)",
                       "note": "the call's time includes its host synchronisation"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "peak_source": f"{src} hbm_gbs"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_factor(args):
    """The mixed path's dense factorisation alone: glasso_cholinv_mixed (FP32
    Cholesky A = L L^T with the inverse factor X = L^-1 formed alongside, then
    W = X^T X, every O(n^3) contraction a split-TF32 tcgen05 product) on an
    iterate-like SPD matrix (S + lambda I of the sparse-Theta generator's
    samples, m = n/2).  value = algorithmic TFLOP/s, n^3 flops per call
    (n^3/3 each for L, X and W)."""
    import torch

    from paper_1607_00315_gb300 import build, glasso, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    n = args.factor_n
    p = synth.random_problem(n, max(n // 2, 2), 0.1, 9100 + n, gen="sparse")
    ctx = glasso.Context(local, precision=glasso.MIXED)
    ctx.set_debug(glasso.DEBUG_TC_DAG_TILES, args.dag_tiles)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    S = torch.empty((n, n), dtype=torch.float64, device=dev)
    glasso.Context(local).form_S(torch.from_numpy(p.X).to(dev), S)
    A = S + 0.1 * torch.eye(n, dtype=torch.float64, device=dev)
    W = torch.empty_like(A)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        info, _ = ctx.cholinv_mixed(A, W)
        assert info == 0
    lat = []
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.cholinv_mixed(A, W)
            e1.record(stream)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
    if args.profile_range:
        torch.cuda.profiler.stop()
    ms = float(np.mean(lat))
    _, bf16, src = peaks()
    peak = tf32_peak_tflops(sustained_bf16(bf16))
    tf = float(n) ** 3 / (ms * 1e-3) / 1e12
    line = {"metric": "dense factorisation + inverse of the mixed path (glasso_cholinv_mixed)",
            "value": tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "split-tf32 (f32 storage)", "data": "synthetic",
            "config": {"workload": f"cholinv_mixed n={n}", "n": n, "dag_tiles": args.dag_tiles,
                       "l2": "flushed between timed calls (512 MB write)"},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak,
                         "peak_source": f"TF32 = {src} bf16 sustained x nominal 1.1/2.25"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="path whose solves/s is `value` (the other one is timed beside it)")
    ap.add_argument("--inner", default="pcd_cg", choices=["cd", "pcd_cg"],
                    help="Newton-direction solver of the single solves (the other is timed beside it): "
                         "PCD-CG, Section 6.3's inner solver, by default")
    ap.add_argument("--batch-inner", default="auto", choices=["cd", "pcd_cg", "auto"],
                    help="Newton-direction solver of the batched and serving workloads (auto by default: per "
                         "relaxation PCD-CG when the CD sweeps' serial chain would be long, CD sweeps when the "
                         "free set is small and PCD-CG's fixed cost would dominate)")
    ap.add_argument("--batch-engine", default="fused", choices=["fused", "slots"],
                    help="batched workload: one persistent launch over all paths (fused) or the host-driven "
                         "serving slots")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other precision path")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end solves through the public API (0: the same as --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (n=10000, batched, serving) reported beside the headline")
    ap.add_argument("--factor-n", type=int, default=2000, help="factor: matrix size")
    ap.add_argument("--dag-tiles", type=int, default=0,
                    help="largest diagonal block (in 128-row tiles) of one task-graph launch of the "
                         "mixed factorisation: 0 the library default, 1 none (plain recursion)")
    ap.add_argument("--scan-n", type=int, default=2000, help="scan: matrix size")
    ap.add_argument("--workload", default="solve", choices=["solve", "batched", "serving", "factor", "scan"],
                    help="solve: the n=2000 single-solve metric (default); batched: lambda paths "
                         "of many small instances; serving: a Poisson request stream; factor: "
                         "the mixed path's tensor-core factorisation alone; scan: the free-set scan alone")
    ap.add_argument("--instances", type=int, default=512, help="batched: instances")
    ap.add_argument("--screen", action="store_true",
                    help="batched: exact screening (isolated vertices in closed form)")
    ap.add_argument("--requests", type=int, default=300, help="serving: requests of the trace")
    ap.add_argument("--rate", type=float, default=60.0,
                    help="serving: arrivals per second (60: the device loaded, not saturated)")
    ap.add_argument("--profile-range", action="store_true",
                    help="open the CUDA profiler range around the timed solves only "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "factor":
        return run_factor(args)
    if args.workload == "scan":
        return run_scan(args)

    import torch
    import torch.distributed as dist

    from paper_1607_00315_gb300 import build, glasso, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    # independent instances per rank (weak scaling, no data-path collective)
    p = synth.config_problem(CONFIG_ID, instance=rank)
    prec = glasso.FP64 if args.precision == "fp64" else glasso.MIXED
    ctx = glasso.Context(local, precision=prec)
    ctx.set_debug(glasso.DEBUG_TC_DAG_TILES, args.dag_tiles)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    # the workload's input is the FP64 covariance S (eq. cov_estimate), formed
    # once on the GPU from the samples, outside the timed region
    S = torch.empty((p.n, p.n), dtype=torch.float64, device=dev)
    glasso.Context(local).form_S(torch.from_numpy(p.X).to(dev), S)
    torch.cuda.synchronize()
    A_out = torch.empty((p.n, p.n), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        _, _, info = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner)
        return info

    for _ in range(max(args.warmup, 3)):
        info = step()
    ctx.set_profiling(True)
    ctx.get_profile(reset=True)
    lat, infos = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict the L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step())
            e1.record(stream)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    prof = ctx.get_profile(reset=True)
    ctx.set_profiling(False)
    A_this = A_out.clone()  # the timed path's solution, for the comparison below
    total_ms, value = job_value(sum(lat), args.steps, world, dev)

    # the other precision path on the same input, same timing protocol
    compare = None
    if not args.no_compare:
        other = glasso.MIXED if prec == glasso.FP64 else glasso.FP64
        octx = glasso.Context(local, precision=other)
        octx.set_stream(stream.cuda_stream)
        oinfo = None
        for _ in range(2):
            _, _, oinfo = octx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner)
        olat = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, oinfo = octx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner)
            e1.record(stream)
            torch.cuda.synchronize()
            olat.append(e0.elapsed_time(e1))
        # the mixed result against the FP64 path's (the FP64 path meets the
        # oracle's bar in the parity tests): reported objective, the objective
        # of the mixed A evaluated in FP64, and the largest entry difference
        if other == glasso.FP64:
            _, F_exact = octx.objective(S, A_this, p.lam)
            F64 = oinfo["objective"]
            Fm = infos[-1]["objective"]
            prec_err = {"objective_fp64_path": F64, "objective_mixed_reported": Fm,
                        "objective_mixed_A_in_fp64": F_exact,
                        "rel_err_reported": abs(Fm - F64) / abs(F64),
                        "rel_err_exact": abs(F_exact - F64) / abs(F64),
                        "max_abs_entry_diff": float((A_this - A_out).abs().max().item()),
                        "note": "both paths stop at rel. KKT 1e-5, so the difference includes "
                                "their different stopping points"}
        else:
            prec_err = None
        octx.close()
        oname = "fp64" if other == glasso.FP64 else "mixed"
        this = "mixed" if prec == glasso.MIXED else "fp64"
        ms = {this: total_ms / args.steps, oname: float(np.mean(olat))}
        compare = {"ms_per_solve": ms, "mixed_speedup_over_fp64": ms["fp64"] / ms["mixed"],
                   "mixed_vs_fp64": prec_err,
                   f"{oname}_solve": {"relaxations": oinfo["relaxations"], "rel_kkt": oinfo["rel_kkt"],
                                      "objective": oinfo["objective"]}}
        # the paper's comparison (Section 8): the ML-cycle against the
        # one-level method (the full free set every cycle) and the one-level
        # method after continuation stages, on the same kernels and input:
        # time, relaxations and the largest support seen (max-supp)
        lv = {}
        for name, one, cont in (("ml_cycle", False, False), ("one_level", True, False),
                                ("continuation", True, True)):
            linfo = None
            for _ in range(2):
                _, _, linfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner, one_level=one,
                                        continuation=cont)
            llat = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, _, linfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner, one_level=one,
                                        continuation=cont)
                e1.record(stream)
                torch.cuda.synchronize()
                llat.append(e0.elapsed_time(e1))
            lv[name] = {"ms_per_solve": float(np.mean(llat)), "relaxations": linfo["relaxations"],
                        "cycles": linfo["cycles"], "max_supp": linfo["max_nnz"], "nnz": linfo["nnz"],
                        "objective": linfo["objective"]}
        compare["levels"] = lv
        # exact screening on the same input: isolated vertices of {|S_ij| > lambda}
        # in closed form, the other vertices as one sub-problem (same minimiser)
        sinfo = None
        for _ in range(2):
            _, _, sinfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner, screen=True)
        slat = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, sinfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=args.inner, screen=True)
            e1.record(stream)
            torch.cuda.synchronize()
            slat.append(e0.elapsed_time(e1))
        compare["screened"] = {"ms_per_solve": float(np.mean(slat)), "components": sinfo["components"],
                               "max_block": sinfo["max_block"], "relaxations": sinfo["relaxations"],
                               "nnz": sinfo["nnz"], "objective": sinfo["objective"]}
        # the Newton-direction solver: CD sweeps against PCD-CG to Section 8's
        # relative precision 1e-4, same input and protocol (the timed one above,
        # the other one here)
        oinner = "pcd_cg" if args.inner == "cd" else "cd"
        pinfo = None
        for _ in range(2):
            _, _, pinfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=oinner)
        plat = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, pinfo = ctx.solve(S, p.lam, tol=p.tol, A_out=A_out, inner=oinner)
            e1.record(stream)
            torch.cuda.synchronize()
            plat.append(e0.elapsed_time(e1))
        compare["inner"] = {
            args.inner: {"ms_per_solve": total_ms / args.steps, "relaxations": infos[-1]["relaxations"],
                         "inner_iters": infos[-1]["inner_iters"], "rel_kkt": infos[-1]["rel_kkt"],
                         "objective": infos[-1]["objective"], "timed": True},
            oinner: {"ms_per_solve": float(np.mean(plat)), "relaxations": pinfo["relaxations"],
                     "inner_iters": pinfo["inner_iters"], "rel_kkt": pinfo["rel_kkt"],
                     "objective": pinfo["objective"], "status": pinfo["status"]}}

    # end to end through the public API with host buffers (pinned): S in, A out
    Sh = S.cpu().pin_memory().numpy()
    Ah = torch.empty((p.n, p.n), dtype=torch.float64).pin_memory().numpy()
    e2e = []
    for _ in range(args.e2e_steps if args.e2e_steps > 0 else args.steps):
        t0 = time.perf_counter()
        ctx.solve(Sh, p.lam, tol=p.tol, A_out=Ah, inner=args.inner)
        e2e.append(time.perf_counter() - t0)
    _, e2e_value = job_value(sum(e2e) * 1e3, len(e2e), world, dev)

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel class, from the live CUDA-event timings;
    # kernels run inside a solve of tens of ms, so the sustained bf16 figure
    hbm, bf16, src = peaks()
    bf16_s = sustained_bf16(bf16)
    classes = {k: v for k, v in prof.items()
               if isinstance(v, dict) and "launches" in v and v["launches"] > 0}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    per_launch_ms = d["ms"] / d["launches"]
    work_per_launch = d["work"] / d["launches"]
    if dom in ("cholesky", "inverse", "ls_cholesky", "ns_refine"):
        achieved = work_per_launch / (per_launch_ms * 1e-3) / 1e12
        if args.precision == "fp64":
            peak = fp64_peak_tflops(bf16_s)
            psrc = f"FP64 = {src} bf16 sustained {bf16_s} TF/s x nominal 1.25/2250"
            bound = "alu"
        else:
            # split-TF32 tensor-core kernels (ns_refine: single TF32); algorithmic
            # flops, so a split product (3 MMAs) can reach at most 1/3 of the peak
            peak = tf32_peak_tflops(bf16_s)
            psrc = f"TF32 = {src} bf16 sustained {bf16_s} TF/s x nominal 1.1/2.25"
            bound = "tensor"
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": psrc}
    else:
        achieved = work_per_launch / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"{src} hbm_gbs"}
    roof["kernel"] = dom
    roof["launch_ms"] = per_launch_ms
    roof["work_per_launch"] = work_per_launch
    roof["traffic"] = ncu_traffic(dom, args.inner if dom == "cd_sweeps" else None)
    share = {k: round(v["ms"] / sum(c["ms"] for c in classes.values()), 4) for k, v in classes.items()}
    # every timed class against its own roofline (the same arithmetic as above)
    per_class = {}
    for k, v in classes.items():
        lm = v["ms"] / v["launches"]
        wk = v["work"] / v["launches"]
        if k in ("scan", "cd_sweeps"):
            a = wk / (lm * 1e-3) / 1e9
            per_class[k] = {"launch_ms": lm, "launches": v["launches"], "achieved": a, "unit": "GB/s",
                            "frac": a / hbm}
        else:
            a = wk / (lm * 1e-3) / 1e12
            pk = fp64_peak_tflops(bf16_s) if args.precision == "fp64" else tf32_peak_tflops(bf16_s)
            per_class[k] = {"launch_ms": lm, "launches": v["launches"], "achieved": a, "unit": "TFLOP/s",
                            "frac": a / pk}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "mixed(f32/tf32+f64)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "n": p.n, "m": p.m, "lambda": p.lam, "tol": p.tol, "input": "S (fp64) given",
                   "precision": args.precision, "inner": args.inner, "dag_tiles": args.dag_tiles,
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat))},
        "solve": {"cycles": infos[-1]["cycles"], "relaxations": infos[-1]["relaxations"],
                  "ls_trials": infos[-1]["ls_trials"], "rel_kkt": infos[-1]["rel_kkt"],
                  "objective": infos[-1]["objective"], "nnz": infos[-1]["nnz"]},
        "time_share": share,
        "class_roofline": per_class,
        "compare": compare,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(Sh.nbytes),
                "d2h_bytes_per_step": int(Ah.nbytes)},
        "gpu_launches": int(prof["kernels"]),
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_extra:
        line["workloads"] = extra_workloads(args, local, dev)
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        ncpu, model = host_cpu()
        t_solve, oinfo = oracle_solve_timed(S.cpu().numpy(), p.lam, p.tol)
        line["cpu_baseline"] = {
            "value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "host_cpus": ncpu, "cpu_model": model,
            "sample": f"one whole FP64 oracle solve of the same S to rel. KKT {p.tol} on one core "
                      f"({t_solve:.2f} s, {oinfo['relaxations']} relaxations, rel. KKT "
                      f"{oinfo['rel_kkt']:.2e})"}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
