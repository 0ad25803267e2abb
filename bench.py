"""Benchmark: kernel-mode PCG obs*iter/s and solves/s on one GB300.

Workload (default): the mixed-precision kernel-mode solve with n = 8,000
Gaussian-RBF points on [0, 1] (bandwidth 0.1), finite modes 400 x 500,
q = 5e7 observations (uniform without replacement, sorted by kernel index),
planted smooth rank-40 model + 1% noise, r = 40, lambda = 1e-4, rho = 1e-6,
tolerance 1e-6 on the FP64 true relative residual.  Synthetic data (seeded).
Operator arithmetic (--precision): mixed_bf16x3, the two n x n products on
the tensor cores from 3 BF16 slices per operand, the gather-dot/scatter in
FP32, FP64 CG scalars and FP64-accurate true residuals.

A step is one subproblem through every step of the path: problem creation
from device-resident inputs (validation, Zhat, row pointer, pieces, Gram,
eig(V), MTTKRP) followed by the PCG solve (right-hand side, iterations,
FP64-accurate true residuals, W = U_K Wbar).  eig(K) is the one-time
per-kernel setup and stays outside the timed region.  Zhat (16 GB as an FP32
pair) is far larger than the 129 MB L2, so no flush is needed between steps.

Besides the headline line's own fields, the same JSON line carries: the FP64
path on the same workload, the other operator arithmetics (--sweep), the
end-to-end rate through the one-shot call with pinned host buffers, a batch
of 256 uneven subproblems submitted at once (--batch), Poisson-arrival
serving (--serve-rates), the alternating fit of the full model (--als-ranks),
the paper's vortex / Miranda shapes (--no-paper-shapes to skip), the FP64
oracle on a bounded sample of the host cores, and nvidia-smi clocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kernel-mode PCG obs*iter/s & solves/s, mixed vs FP64 at 1e-6 rel err; p50/p99"
UNIT = "obs*iter/s"
WORKLOAD = "c3_mixed_n8000_q5e7_r40"
TOL = 1e-6
# DRAM bytes (read + write) per observation of the FP32 gather-dot/scatter
# launch at r = 40, from one ncu capture of the same kernel at n = 2000,
# q = 5e6 (810.0 MB read + 3.6 MB written per launch); traffic grows in
# proportion to q.
GDS32_TRAFFIC_PER_OBS_R40 = 813.6e6 / 5e6
MAX_ITER_BATCH = 5000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="mixed_bf16x3",
                    help="operator arithmetic of the single-solve workload")
    ap.add_argument("--batch-precision", default="mixed_fp32",
                    help="operator arithmetic of the batched and served subproblems (n <= 2000 "
                         "but for the large served requests; the persistent launch is FP32)")
    ap.add_argument("--sweep",
                    default="mixed_fp32,mixed_bf16x3,mixed_tf32x3,mixed_tf32,mixed_bf16,"
                            "fp64_emulated",
                    help="other operator arithmetics timed on the same data (2 steps each)")
    ap.add_argument("--q", type=int, default=0, help="override q (smaller runs)")
    ap.add_argument("--n", type=int, default=0, help="override n (smaller runs)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=256,
                    help="uneven subproblems in the batched run (0: skip)")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000",
                    help="Poisson arrival rates (req/s) of the serving run ('' : skip)")
    ap.add_argument("--serve-fp64-rates", default="50,200",
                    help="rates at which the FP64 one-at-a-time path is also served")
    ap.add_argument("--slots", type=int, default=16, help="requests running at once")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the autotuned batch run")
    ap.add_argument("--als-ranks", default="10,20,40",
                    help="ranks of the alternating-fit run (n=2000, 200x300, q=6e6; '' : skip)")
    ap.add_argument("--als-sweeps", type=int, default=20)
    ap.add_argument("--no-paper-shapes", action="store_true",
                    help="skip the runs on the paper's vortex / Miranda shapes")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per serving rate (at most --serve-seconds of arrivals)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--no-gram", dest="gram", action="store_false",
                    help="skip the compressed-Gram runs")
    ap.add_argument("--tol2", type=float, default=1e-8,
                    help="second tolerance of the single-solve workload (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(world, device, sums, maxes):
    """Whole-job aggregation of independent replicas: `sums` are added over
    the ranks (units processed), `maxes` take the slowest rank (times).  With
    one rank the values are returned as they are."""
    sums, maxes = [float(x) for x in sums], [float(x) for x in maxes]
    if world == 1:
        return sums, maxes
    import torch
    import torch.distributed as dist
    t = torch.tensor(sums, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    u = torch.tensor(maxes, dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.MAX)
    return t.tolist(), u.tolist()


def replica_seed(rank: int, base: int = 0) -> int:
    """Seed of rank `rank`'s independent subproblem (replicas only: no data
    is exchanged between ranks)."""
    return base + rank


def config_dict(args, p, world):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": args.workload, "n": p.n, "other_sizes": p.other_sizes, "q": p.q,
            "r": p.r, "lambda": p.lam, "rho": p.rho, "tol": TOL, "precision": args.precision,
            "values": "fp32", "indices": "int32, sorted by kernel index",
            "parallelism": f"replicas x{world}", "l2": "inputs larger than L2"}


def make_problem(args, seed):
    import synth
    over = {}
    if args.q:
        over["q"] = args.q
    if args.n:
        over["n"] = args.n
    return synth.workload(args.workload, seed=seed, **over)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # sampling has started when the timed region begins
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_setup(p, sample_q: int):
    """Oracle operators on the first `sample_q` sorted observations (setup,
    untimed: Zhat, Gram, eig(K) and eig(V), right-hand side)."""
    import oracle as O
    q = min(sample_q, p.q)
    kidx, oidx, vals = p.kidx[:q], p.oidx[:q], p.vals[:q]
    Zh = O.zhat(p.factors, oidx)
    V = O.gram(p.factors)
    g = O.density(p.n, p.other_sizes, q)
    UK, UV, D = O.precond_setup(p.K, V, g, p.lam, p.rho)
    b = p.K @ O.mttkrp(p.n, kidx, vals, Zh)
    A = lambda X: O.matvec(p.K, kidx, Zh, p.lam, p.rho, X)
    Minv = lambda R: O.precond_apply(UK, UV, D, R)
    return A, Minv, b, q


def cpu_oracle_time(setup, iters: int = 1):
    """Seconds for `iters` oracle PCG iterations (operator + preconditioner)."""
    import oracle as O
    A, Minv, b, q = setup
    t0 = time.perf_counter()
    O.pcg(A, b, Minv, tol=0.0, maxit=iters)
    return time.perf_counter() - t0, q, iters


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    p = make_problem(args, seed=0)
    sample_q = int(os.environ.get("CPHIFI_CPU_SAMPLE_Q", "2000000"))
    setup = cpu_oracle_setup(p, sample_q)
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_time(setup)
    secs, obs = 0.0, 0
    for _ in range(args.steps):
        s, q, it = cpu_oracle_time(setup)
        secs += s
        obs += q * it
    v = obs / secs
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic planted low rank (seeded)",
            "config": config_dict(args, p, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one FP64 oracle PCG iteration (NumPy) per step on the "
                                       f"first {min(sample_q, p.q)} sorted observations, full n"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(args, pkg, ctx, kern, p):
    """Same metric through cphifi_solve with pinned HOST buffers: the H2D copy
    of the inputs and the D2H copy of W are inside the timed region."""
    import torch
    n, r, q = p.n, p.r, p.q
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    kh, oh, vh = pin(p.kidx), pin(p.oidx.ravel()), pin(p.vals.astype(np.float32))
    fh = [pin(np.asfortranarray(F).ravel(order="F")).reshape(F.shape[1], F.shape[0]).T
          for F in p.factors]
    Wh = pin(np.zeros((r, n))).T
    # twice the device-resident steps: an occasional slow call (creations of
    # 50-60 ms instead of 6 ms have been seen, not caused by the library's
    # allocations, which take under a millisecond) then weighs less in the mean
    e2e_steps = max(1, 2 * args.steps)
    # one untimed call first: the context's memory pool then holds the blocks
    # a call needs, as it does in a long-running user process
    pkg.solve(ctx, kern, fh, kh, oh, vh, r, p.lam, p.rho, TOL, 500, precision=args.precision,
              sorted_obs=True, out=Wh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    host_setup_ms, host_solve_ms = [], []
    for _ in range(e2e_steps):
        Wo, st = pkg.solve(ctx, kern, fh, kh, oh, vh, r, p.lam, p.rho, TOL, 500,
                           precision=args.precision, sorted_obs=True, out=Wh)
        e2e_iters += st["iterations"]
        host_setup_ms.append(st["setup_ms"])
        host_solve_ms.append(st["solve_ms"])
    torch.cuda.synchronize()
    te2e = time.perf_counter() - t0
    h2d = q * 4 + q * 4 * p.oidx.shape[1] + q * 4 + sum(F.size * 8 for F in p.factors)
    return {"value": q * e2e_iters / te2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(n * r * 8), "solves_per_s": e2e_steps / te2e,
            "host_create_ms": host_setup_ms, "host_solve_ms": host_solve_ms}


class BatchInputs:
    """Device-resident inputs of uneven subproblems and their kernels (eig(K)
    is the one-time per-kernel setup: computed here, outside any timing)."""

    def __init__(self, pkg, ctx, dev, specs):
        import torch
        import synth
        self.specs = specs
        self.kerns = {}
        self.items = []
        for sp in specs:
            p = synth.batch_problem(sp)
            key = (p.n, sp["kernel"])
            if key not in self.kerns:
                dK, UK = np.linalg.eigh(p.K)
                self.kerns[key] = ctx.kernel_create(p.n, UK, dK)
            self.items.append(self.upload(p, self.kerns[key], dev))

    @staticmethod
    def upload(p, kern, dev):
        import torch
        return dict(
            p=p, kern=kern, q=p.q, n=p.n, r=p.r,
            f=[torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors],
            k=torch.from_numpy(p.kidx).to(dev),
            o=torch.from_numpy(np.ascontiguousarray(p.oidx).ravel()).to(dev),
            v=torch.from_numpy(p.vals).to(dev),
            W=torch.empty(p.n * p.r, dtype=torch.float64, device=dev))

    def close(self):
        for k in self.kerns.values():
            k.close()


def submit_item(pkg, ctx, it, precision):
    p = it["p"]
    return pkg.submit(ctx, it["kern"], it["f"], it["k"], it["o"], it["v"], p.r, p.lam, p.rho, TOL,
                      max_iter=MAX_ITER_BATCH, precision=precision, sorted_obs=True,
                      out=it["W"])


def _timed_batch(pkg, ctx, items, precision):
    """Submits every item at once and waits for all: (elapsed s, stats, completion
    times by ticket, requests)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reqs = [submit_item(pkg, ctx, it, precision) for it in items]
    done_t = {}
    while len(done_t) < len(reqs):
        _, _, done = ctx.poll(done_cap=64)
        now = time.perf_counter()
        for t in done:
            done_t[t] = now
    res = [r_.wait() for r_ in reqs]
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    stats = [st for _, st in res]
    lat = sorted(1e3 * (done_t[r_.ticket] - t0) for r_ in reqs)
    pct = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
    launches = sum(st["kernel_launches"] + st["setup_launches"] for st in stats)
    obs_iter = sum(it["q"] * st["iterations"] for it, st in zip(items, stats))
    return {"elapsed_ms": 1e3 * elapsed, "solves_per_s": len(items) / elapsed,
            "obs_iter_per_s": obs_iter / elapsed,
            "converged": sum(1 for st in stats if st["status"] == 0),
            "max_rel_residual": max(st["rel_residual"] for st in stats),
            "completion_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": lat[-1]},
            "gpu_launches": int(launches), "launches_per_solve": launches / len(items),
            "host_create_ms_sum": sum(st["setup_ms"] for st in stats),
            "iterations": int(sum(st["iterations"] for st in stats))}


def _timed_persistent(pkg, ctx, items):
    """cphifi_solve_batch over every item: the problems created on the
    library's streams, then one persistent launch for all solves.  Host clock
    around the call (it returns with the results written)."""
    import torch
    probs = [dict(kernel=it["kern"], factors=it["f"], kidx=it["k"], oidx=it["o"], vals=it["v"],
                  r=it["r"], sorted_obs=True, out=it["W"]) for it in items]
    p0 = items[0]["p"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, stats, info = pkg.solve_batch(ctx, probs, p0.lam, p0.rho, TOL, max_iter=MAX_ITER_BATCH)
    elapsed = time.perf_counter() - t0
    lat = sorted(st["iter_ms"] for st in stats)  # launch start -> each solve's completion
    pct = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
    obs_iter = sum(it["q"] * st["iterations"] for it, st in zip(items, stats))
    launches = sum(st["setup_launches"] for st in stats) + 1
    return {"elapsed_ms": 1e3 * elapsed, "solves_per_s": len(items) / elapsed,
            "obs_iter_per_s": obs_iter / elapsed,
            "converged": sum(1 for st in stats if st["status"] == 0),
            "max_rel_residual": max(st["rel_residual"] for st in stats),
            "kernel_ms": info["kernel_ms"], "create_ms": info["create_ms"],
            "solves_per_s_kernel": len(items) / (1e-3 * info["kernel_ms"]),
            "completion_in_launch_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": lat[-1]},
            "tiles": info["tiles"], "blocks": info["blocks"], "timed_out": info["timed_out"],
            "gpu_launches": int(launches), "launches_per_solve": launches / len(items),
            "iterations": int(sum(st["iterations"] for st in stats))}


def run_batch(args, pkg, ctx, dev, seed):
    """All subproblems at once, two ways.  (1) Submitted: every request's PCG
    runs on its own stream, each chunk of iterations replayed from a CUDA
    graph, as slots and HBM free up; timed on the host clock from the first
    submit to the last completion, with the device idle on both sides, then
    again after the autotuner has chosen the launch shapes of the batch's
    size buckets (untimed).  (2) Persistent: cphifi_solve_batch, every solve
    in one kernel launch (best of two calls)."""
    import torch
    import synth
    B = BatchInputs(pkg, ctx, dev, synth.batch_specs(seed, args.batch))
    items = B.items
    for it in items[:16]:  # warm-up: module loads, pools, pinned slots
        submit_item(pkg, ctx, it, args.batch_precision).wait()
    untuned = _timed_batch(pkg, ctx, items, args.batch_precision)
    tuned = None
    if args.autotune:
        from paper_2603_25691_gb300 import autotune
        cache = autotune.Cache(None)
        t0 = time.perf_counter()
        insts = [(it["kern"], dict(factors=it["f"], kidx=it["k"], oidx=it["o"], vals=it["v"],
                                   r=it["r"], lam=it["p"].lam, rho=it["p"].rho, sorted=True))
                 for it in items]
        nb = cache.tune_instances(ctx, insts, args.batch_precision, iters=6, reps=1)
        tune_s = time.perf_counter() - t0
        cache.apply(ctx, args.batch_precision)
        for it in items[:16]:
            submit_item(pkg, ctx, it, args.batch_precision).wait()
        tuned = _timed_batch(pkg, ctx, items, args.batch_precision)
        tuned.update({"buckets_tuned": nb, "tuning_s": tune_s})
    persistent = None
    for _ in range(2):
        run = _timed_persistent(pkg, ctx, items)
        if persistent is None or run["elapsed_ms"] < persistent["elapsed_ms"]:
            persistent = run
    # The plain FP64 GPU path, one subproblem at a time, same inputs and tolerance.
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    it64 = 0
    for it in items:
        p = it["p"]
        _, st = pkg.solve(ctx, it["kern"], it["f"], it["k"], it["o"], it["v"], p.r, p.lam, p.rho,
                          TOL, max_iter=MAX_ITER_BATCH, precision="fp64", sorted_obs=True,
                          out=it["W"])
        it64 += st["iterations"]
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t1
    best = tuned if tuned and tuned["elapsed_ms"] < untuned["elapsed_ms"] else untuned
    if persistent["converged"] == len(items) and persistent["elapsed_ms"] < best["elapsed_ms"]:
        best = persistent
    out = {"workload": f"c4_batch_{len(items)}_uneven", "precision": args.batch_precision,
           "tol": TOL,
           "requests": len(items), "sum_q": int(sum(it["q"] for it in items)),
           "n_grid": list(synth.BATCH_N_GRID), "kernels": len(B.kerns), **untuned,
           "autotuned": tuned, "persistent": persistent,
           "fp64_one_at_a_time": {"solves_per_s": len(items) / t64, "elapsed_ms": 1e3 * t64,
                                  "iterations": it64},
           "speedup_vs_fp64_one_at_a_time": t64 / (best["elapsed_ms"] / 1e3),
           "slots": args.slots}
    B.close()
    return out


def _pcts(lat):
    lat = sorted(lat)
    if not lat:
        return {"p50_ms": None, "p99_ms": None, "max_ms": None, "count": 0}
    pct = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
    return {"p50_ms": pct(0.5), "p99_ms": pct(0.99), "max_ms": lat[-1], "count": len(lat)}


def run_serve(args, pkg, ctx, dev, seed, big_kern, big_p):
    """Poisson arrivals of subproblems sized as the batch (plus 5% large ones,
    n = 8000, q = 2e7, r = 40); each is submitted at its arrival time and its
    latency runs from the arrival to the poll that sees it complete.  At the
    rates of --serve-fp64-rates the same arrivals are also served by the plain
    FP64 path one request at a time (cphifi_solve in arrival order)."""
    import torch
    import synth
    rates = [float(x) for x in args.serve_rates.split(",") if x]
    rates64 = {float(x) for x in args.serve_fp64_rates.split(",") if x}
    pool = BatchInputs(pkg, ctx, dev, synth.batch_specs(seed + 7, 64))
    big = BatchInputs.upload(big_p, big_kern, dev) if big_p is not None else None
    rng = np.random.default_rng(seed)
    out = []
    for it in pool.items[:8]:
        submit_item(pkg, ctx, it, args.batch_precision).wait()
    if big is not None:  # the large shape once alone: its latency on an idle GPU
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        submit_item(pkg, ctx, big, args.batch_precision).wait()
        big_alone_ms = 1e3 * (time.perf_counter() - t0)
    for rate in rates:
        nreq = int(min(args.serve_requests, max(20, args.serve_seconds * rate)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
        which = [big if (big is not None and rng.uniform() < 0.05) else
                 pool.items[int(rng.integers(len(pool.items)))] for _ in range(nreq)]
        # distinct output buffers: requests in flight may share an instance
        outs = [torch.empty_like(it["W"]) for it in which]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        tick = {}
        done_t = {}
        while len(done_t) < nreq:
            now = time.perf_counter() - t0
            while k < nreq and arrivals[k] <= now:
                it = dict(which[k])
                it["W"] = outs[k]
                rq = submit_item(pkg, ctx, it, args.batch_precision)
                tick[rq.ticket] = (k, rq)
                k += 1
            _, _, done = ctx.poll(done_cap=256)
            now = time.perf_counter() - t0
            for t in done:
                done_t[tick[t][0]] = now
        sts = {i: rq.wait()[1] for i, rq in tick.values()}
        lat = [1e3 * (done_t[i] - arrivals[i]) for i in range(nreq)]
        is_big = [it is big for it in which]
        span = max(done_t.values()) - arrivals[0]
        row = {"rate_req_s": rate, "requests": nreq, "large": int(sum(is_big)),
               "solves_per_s": nreq / span, **_pcts(lat),
               "small": _pcts([x for x, b in zip(lat, is_big) if not b]),
               "large_lat": _pcts([x for x, b in zip(lat, is_big) if b]),
               "mean_queue_ms": float(np.mean([sts[i]["queue_ms"] for i in range(nreq)])),
               "converged": sum(1 for st in sts.values() if st["status"] == 0)}
        if rate in rates64:
            # the plain FP64 GPU path, one request at a time in arrival order
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat64 = []
            for i, it in enumerate(which):
                now = time.perf_counter() - t0
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                pp = it["p"]
                pkg.solve(ctx, it["kern"], it["f"], it["k"], it["o"], it["v"], pp.r, pp.lam,
                          pp.rho, TOL, max_iter=MAX_ITER_BATCH, precision="fp64",
                          sorted_obs=True, out=outs[i])
                lat64.append(1e3 * (time.perf_counter() - t0 - arrivals[i]))
            span64 = time.perf_counter() - t0 - arrivals[0]
            row["fp64_one_at_a_time"] = {"solves_per_s": nreq / span64, **_pcts(lat64)}
        out.append(row)
    pool.close()
    return {"rates": out, "large_alone_ms": big_alone_ms if big is not None else None,
            "slots": args.slots}


# Stand-ins for the paper's unaligned experiments (§5.2): mode sizes of the
# vortex (199 x 449 x 151, Gaussian sigma = (4, 4, 3)) and Miranda (256 x 256
# x 269, sigma = (1, 1, 2)) tensors on integer grids, q = 50,000 uniform
# observations, lambda = 0.1, rho = 1e-6, tol 1e-6, at most 75 iterations,
# r in {5, 10, ..., 50}.  The data values are planted (the datasets are not
# available).  Each mode in turn is the kernel mode, the other two finite.
PAPER_SHAPES = {"vortex": ((199, 449, 151), (4.0, 4.0, 3.0)),
                "miranda": ((256, 256, 269), (1.0, 1.0, 2.0))}


def run_paper_shapes(args, pkg, ctx, seed):
    import synth
    out = {}
    for name, (dims, sig) in PAPER_SHAPES.items():
        rows = []
        for k in range(3):
            n = dims[k]
            other = tuple(dims[m] for m in range(3) if m != k)
            x = synth.grid_points(n, integer=True)
            K = synth.gaussian_kernel(x, sig[k])
            dK, UK = np.linalg.eigh(K)
            kern = ctx.kernel_create(n, UK, dK)
            for r in range(5, 51, 5):
                p = synth.planted_problem(seed + 97 * k + r, n, other, 50_000, r, bandwidth=sig[k],
                                          integer_grid=True, lam=0.1, rho=1e-6)
                for prec in ("fp64", "mixed_fp32"):
                    t0 = time.perf_counter()
                    W, st = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, r, p.lam,
                                      p.rho, 1e-6, 75, precision=prec, sorted_obs=True)
                    ms = 1e3 * (time.perf_counter() - t0)
                    rows.append({"mode": k, "n": n, "r": r, "precision": prec, "ms": ms,
                                 "iterations": st["iterations"], "status": st["status"],
                                 "rel_residual": st["rel_residual"]})
            kern.close()
        summ = {}
        for prec in ("fp64", "mixed_fp32"):
            sel = [x for x in rows if x["precision"] == prec]
            summ[prec] = {"solves": len(sel), "mean_ms": float(np.mean([x["ms"] for x in sel])),
                          "max_ms": float(np.max([x["ms"] for x in sel])),
                          "converged": int(sum(1 for x in sel if x["status"] == 0)),
                          "max_iterations": int(max(x["iterations"] for x in sel)),
                          "sweep_ms_r25": float(sum(x["ms"] for x in sel if x["r"] == 25))}
        out[name] = {"dims": dims, "sigma": sig, "q": 50_000, "lambda": 0.1, "rho": 1e-6,
                     "tol": 1e-6, "max_iter": 75, "summary": summ}
    return out


def run_als(args, pkg, ctx, seed):
    """The full alternating fit (§2) on the device: kernel mode n = 2000
    (Gaussian, bandwidth 0.1), finite modes 200 x 300 updated by CP-ALS rows,
    q = 6e6 planted observations, lambda = 1e-4, a fixed number of sweeps
    from a random start; kernel-mode PCG in FP64 to 1e-6 with at most 75
    iterations (the paper's §5 settings).  Timed on the host clock around
    cphifi_als with host inputs (their upload and the model's download
    included); eig(K) is the one-time setup outside."""
    import synth
    out = []
    p = synth.workload("c2_fp64_n2000_q6e6_r20", seed=seed)
    dK, UK = np.linalg.eigh(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    for r in [int(x) for x in args.als_ranks.split(",") if x]:
        rng = np.random.default_rng(seed + r)
        start = [rng.standard_normal((F.shape[0], r)) for F in p.factors]
        # warm-up: one sweep (module loads, pools)
        pkg.als(ctx, kern, start, p.kidx, p.oidx, p.vals, r, p.lam, p.rho, tol=1e-6,
                sweeps=1, max_iter=75, precision="fp64", sorted_obs=True)
        t0 = time.perf_counter()
        W, facs, errs, st = pkg.als(ctx, kern, start, p.kidx, p.oidx, p.vals, r, p.lam, p.rho,
                                    tol=1e-6, sweeps=args.als_sweeps, max_iter=75,
                                    precision="fp64", sorted_obs=True)
        secs = time.perf_counter() - t0
        out.append({"workload": f"c2_als_n2000_200x300_q6e6_r{r}", "r": r,
                    "sweeps": int(len(errs)), "seconds": secs,
                    "ms_per_sweep": 1e3 * secs / max(1, len(errs)),
                    "fit_error_first": float(errs[0]), "fit_error_last": float(errs[-1]),
                    "precision": "fp64", "pcg_tol": 1e-6, "pcg_max_iter": 75,
                    "last_solve_iterations": st["iterations"]})
    kern.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2603_25691_gb300 as pkg

    # ---- inputs (each rank: its own independent subproblem; replicas only)
    p = make_problem(args, seed=replica_seed(rank))
    dK, UK = np.linalg.eigh(p.K)
    n, r, q = p.n, p.r, p.q
    dev = torch.device("cuda", local)
    kidx_d = torch.from_numpy(p.kidx).to(dev)
    oidx_d = torch.from_numpy(np.ascontiguousarray(p.oidx).ravel()).to(dev)
    vals_d = torch.from_numpy(p.vals.astype(np.float32)).to(dev)  # the workload's FP32 values
    fac_d = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
    W_d = torch.empty(n * r, dtype=torch.float64, device=dev)

    ctx = pkg.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    kern = ctx.kernel_create(n, UK, dK)
    ctx.set_slots(args.slots)

    def step(precision, profile=False, device=True):
        lowp = precision != "fp64"
        if device:
            prob = pkg.Problem(ctx, kern, fac_d, kidx_d, oidx_d, vals_d, r, sorted_obs=True,
                               lowp=lowp)
            W, st = prob.solve(p.lam, p.rho, TOL, max_iter=500, precision=precision,
                               profile=profile, out=W_d, raise_on_error=False)
            prob.close()
        return st

    # ---- warm-up
    for _ in range(args.warmup):
        st = step(args.precision)
    # ---- timed region (device-resident inputs)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stats = []
    step_ms = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev0.record(stream)
        evs[0].record(stream)
        for k in range(args.steps):
            stats.append(step(args.precision, profile=True))
            evs[k + 1].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    iters = sum(s["iterations"] for s in stats)
    iter_phase_ms = sum(s["iter_ms"] for s in stats)
    # The metric: observations x PCG iterations per second of iteration phase
    # (operator, updates, preconditioner, FP64 true residuals and restarts),
    # summed over all ranks' independent problems, over the slowest rank's time.
    (job_obs_iter, job_solves), (elapsed_ms, iter_phase_ms) = reduce_over_ranks(
        world, dev, [q * iters, args.steps], [elapsed_ms, iter_phase_ms])
    value = job_obs_iter / (iter_phase_ms / 1e3)
    solves_per_s = job_solves / (elapsed_ms / 1e3)
    gds_ms = sum(s["gds_ms"] for s in stats)
    gds_bytes_per_launch = q * r * 4 + 2 * n * r * 4  # Zhat (FP32 part) + Xhat rows + Yhat1
    gds_exec = iters
    achieved = gds_bytes_per_launch * gds_exec / (gds_ms / 1e3) / 1e9 if gds_ms > 0 else None
    peak, peak_kind = peaks()
    srt = sorted(step_ms)
    pct = lambda f: srt[min(len(srt) - 1, int(round(f * (len(srt) - 1))))]

    # ---- FP64 path on the same workload (the plain FP64 GPU solve)
    fp64 = None
    if not args.no_fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = step("fp64", profile=True)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        fp64 = {"solves_per_s": 1.0 / t64,
                "obs_iter_per_s": q * s64["iterations"] / (s64["iter_ms"] / 1e3),
                "iterations": s64["iterations"], "rel_residual": s64["rel_residual"],
                "status": s64["status"]}

    # ---- the other operator arithmetics on the same problem (tensor cores etc.)
    sweep = {}
    for prec in [x for x in args.sweep.split(",") if x and x not in ("none", args.precision)]:
        sts = [step(prec, profile=True) for _ in range(1)]   # warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sts = [step(prec, profile=True) for _ in range(2)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        it = sum(x["iterations"] for x in sts) / 2
        itms = sum(x["iter_ms"] for x in sts) / 2
        gm = sum(x["gemm_ms"] for x in sts)
        gl = 2 * sum(x["iterations"] for x in sts)  # executed products (2 per iteration)
        sweep[prec] = {"value": q * it / (itms / 1e3), "solves_per_s": 1e3 / ms,
                       "iterations": it, "iter_phase_ms": itms,
                       "rel_residual": sts[-1]["rel_residual"], "status": sts[-1]["status"],
                       "gemm_avg_ms": gm / max(1, gl)}

    # ---- the same workload at the second tolerance (C3: errors at 1e-6 and 1e-8)
    tol2 = None
    if args.tol2 > 0:
        def step2(precision):
            prob = pkg.Problem(ctx, kern, fac_d, kidx_d, oidx_d, vals_d, r, sorted_obs=True,
                               lowp=precision != "fp64")
            W, st = prob.solve(p.lam, p.rho, args.tol2, max_iter=500, precision=precision,
                               profile=True, out=W_d, raise_on_error=False)
            prob.close()
            return st
        tol2 = {}
        for prec in dict.fromkeys([args.precision, "mixed_fp32", "mixed_tf32x3"]):
            step2(prec)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts = [step2(prec) for _ in range(2)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 2
            it2 = sum(x["iterations"] for x in sts) / 2
            tol2[prec] = {"tol": args.tol2, "solves_per_s": 1e3 / ms, "iterations": it2,
                          "value": q * it2 / (sum(x["iter_ms"] for x in sts) / 2 / 1e3),
                          "true_residuals": sts[-1]["true_residuals"],
                          "rel_residual": sts[-1]["rel_residual"], "status": sts[-1]["status"]}

    # ---- the compressed-Gram form of the product (per-index blocks C_i,
    # Yhat1(i,:) = C_i Xhat(i,:)'): gram = 1 (iterations through FP32 blocks,
    # the FP64-accurate checks stream Zhat) and gram = 2 (checks through
    # FP64-accurate blocks too).  Each step creates the problem, so the blocks'
    # build is inside every timed solve (in the right-hand-side phase).
    gram_runs = None
    if args.gram:
        gram_runs = {}
        for g in (1, 2):
            def stepg():
                prob = pkg.Problem(ctx, kern, fac_d, kidx_d, oidx_d, vals_d, r, sorted_obs=True,
                                   lowp=True)
                W, st = prob.solve(p.lam, p.rho, TOL, max_iter=500, precision=args.precision,
                                   profile=True, out=W_d, raise_on_error=False, gram=g)
                prob.close()
                return st
            stepg()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts = [stepg() for _ in range(2)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 2
            itg = sum(x["iterations"] for x in sts) / 2
            apply_ms = sum(x["gds_ms"] for x in sts) / max(1, sum(x["gds_launches"] for x in sts))
            bytes_apply = n * r * r * 4 + 2 * n * r * 4   # FP32 blocks + Xhat and Yhat1 rows
            gram_runs[f"gram{g}"] = {
                "solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": itg,
                "value": q * itg / (sum(x["iter_ms"] for x in sts) / 2 / 1e3),
                "iter_phase_ms": sum(x["iter_ms"] for x in sts) / 2,
                "ms_per_iteration": sum(x["iter_ms"] for x in sts) / 2 / max(itg, 1),
                "rhs_and_block_build_ms": sum(x["rhs_ms"] for x in sts) / 2,
                "true_residual_ms": sum(x["gds64_ms"] + x["gemm64_ms"] for x in sts) / 2,
                "rel_residual": sts[-1]["rel_residual"], "status": sts[-1]["status"],
                "apply_roofline": {"bound": "hbm", "bytes_per_launch": bytes_apply,
                                   "avg_launch_ms": apply_ms,
                                   "achieved": bytes_apply / (apply_ms / 1e3) / 1e9
                                   if apply_ms > 0 else None,
                                   "peak": peaks()[0], "unit": "GB/s",
                                   "frac": (bytes_apply / (apply_ms / 1e3) / 1e9) / peaks()[0]
                                   if apply_ms > 0 else None}}

    # ---- end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, pkg, ctx, kern, p)

    # ---- batched uneven subproblems, then a served Poisson stream
    batched = None
    if args.batch > 0:
        batched = run_batch(args, pkg, ctx, dev, seed=1000 + rank)
    serving = None
    if args.serve_rates:
        import synth
        big_p = None
        if n == 8000 and p.r == 40:
            big_p = synth.planted_problem(2000 + rank, 8000, (400, 500), 20_000_000, 40,
                                          bandwidth=0.1)
        serving = run_serve(args, pkg, ctx, dev, 3000 + rank, kern if big_p else None, big_p)

    # ---- the paper's unaligned experiment shapes (one-shot solves, host inputs)
    paper = None
    if not args.no_paper_shapes:
        paper = run_paper_shapes(args, pkg, ctx, seed=5000 + rank)

    # ---- the alternating fit (kernel mode + finite modes), FP64
    als_runs = None
    if args.als_ranks:
        als_runs = run_als(args, pkg, ctx, seed=4000 + rank)

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample_q = int(os.environ.get("CPHIFI_CPU_SAMPLE_Q", "2000000"))
        secs, sq, it = cpu_oracle_time(cpu_oracle_setup(p, sample_q), iters=2)
        cpu = {"value": sq * it / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one FP64 oracle PCG iteration (NumPy, BLAS threads = host cores) on "
                         f"the first {sq} sorted observations of this workload, full n = {n}"}
    launches = sum(s["kernel_launches"] + s["setup_launches"] for s in stats)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed_tf32": "tf32 products + f32 gather, f64 CG, df64 residuals",
                      "mixed_bf16": "bf16 products + f32 gather, f64 CG, df64 residuals",
                      "mixed_tf32x3": "3-term split-tf32 products + f32 gather, f64 CG, df64 residuals",
                      "mixed_bf16x3": "bf16x3 products + f32 gather, f64 CG, df64 residuals",
                      "mixed_fp32": "f32 operator, f64 CG, df64 residuals",
                      "fp64_emulated": "df64 (fp32-pair) operator, f64 CG",
                      "fp64": "f64"}[args.precision],
            "data": "synthetic planted low rank (seeded), inputs larger than L2 (no flush)",
            "config": config_dict(args, p, world),
            "solves_per_s": solves_per_s,
            "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "steps": step_ms},
            "step_obs_iter_per_s": job_obs_iter / (elapsed_ms / 1e3),
            "iterations_per_solve": iters / args.steps,
            "rel_residual": [s["rel_residual"] for s in stats],
            "phases_ms_per_solve": {
                "setup": (elapsed_ms / args.steps) - sum(s["rhs_ms"] + s["iter_ms"] + s["final_ms"] for s in stats) / args.steps,
                "rhs": sum(s["rhs_ms"] for s in stats) / args.steps,
                "iteration": iter_phase_ms / args.steps,
                "final": sum(s["final_ms"] for s in stats) / args.steps,
                # inside the iteration phase (CUDA events around each launch):
                "iter_gds": sum(s["gds_ms"] for s in stats) / args.steps,
                "iter_products": sum(s["gemm_ms"] for s in stats) / args.steps,
                "iter_true_residual_gds": sum(s["gds64_ms"] for s in stats) / args.steps,
                "iter_true_residual_products": sum(s["gemm64_ms"] for s in stats) / args.steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": (GDS32_TRAFFIC_PER_OBS_R40 * q
                                     if r == 40 and args.precision in ("mixed_fp32", "mixed_bf16x3")
                                     else None),
                         "kernel": "gds_kernel<float> (gather-dot/scatter, Eqs. vl/yhat1)",
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "bytes_per_launch": gds_bytes_per_launch,
                         "avg_launch_ms": gds_ms / max(1, gds_exec)},
            "fp64_path": fp64,
            "precision_sweep": sweep,
            "second_tolerance": tol2,
            "compressed_gram": gram_runs,
            "mixed_vs_fp64_solves": (solves_per_s / fp64["solves_per_s"]) if fp64 else None,
            "batched": batched, "serving": serving, "als": als_runs, "paper_shapes": paper,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    kern.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
