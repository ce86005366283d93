"""Benchmark: one step = the whole PHS hot path on the tps_1m workload
(n = 1,048,576 points, 90% uniform + 10% in 50 tight clusters, k = 2, linear
block, Vecchia m = 30), i.e. plan creation (normalisation, Morton sort,
quadtree and lists, QR of B, Vecchia enumeration, neighbours and local factors),
the preconditioned CG fit to a 1e-8 relative residual, and evaluation of the
interpolant at 10,000 held-out targets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl native|reference]

Prints one JSON line.  `value` is the device-timed wall time of one step (inputs
resident in HBM, CUDA events on the library's stream, L2 flushed between
steps); `e2e` is the same step through phs_fit_predict_host from host buffers.
For N > 1 (torchrun) every rank runs an independent replica on its own GPU;
`value` is the max over ranks and `fits_per_s` the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG fit time to 1e-8 at n=1M TPS"
WORKLOAD = "tps_1m"
# Preconditioner covariance: Matern nu = 1 in the normalised frame [-1/4,1/4]^2 (Sec. 2.2:
# the nu = 1 kernel carries the thin-plate term, Eq. 2.17).  alpha is the tuning knob of
# Sec. 2.2 (the paper settles on 0.35 for its sets).  ALPHA is what phs_tune_alpha
# returns on another draw of this recipe (seed TUNE_SEED; `--case tune` repeats the
# search): 0.01107, rounded.  On the bench's own draw it needs 11 PCG iterations against
# 12 at 0.03 and 14 at the library default 0.35.  nu = 1.5 converges within 200
# iterations for no alpha of the search (0.035 to 3.5).
NU, ALPHA = 1.0, 0.011
TUNE_SEED = 2002
# k = 3 (cubic workload and the serving stream's k = 3 requests): phs_tune_alpha on another
# draw of the cubic recipe (seed 2003, all 100,000 points) found alpha = 1.005 (40 PCG
# iterations on the bench's own draw against 63 at the library's 0.35), and on held-out
# serving requests (seed 2005, eight k = 3 requests of 48k-495k points) 1.0 took the fewest
# iterations of {0.1, 0.35, 1, 2, 4}; for k = 1 and 2 the library's 0.35 was already best
# there (within 5%), so those keep it.  The count is sensitive near there on the cubic
# draw (47 iterations at 1.0, 53 at 1.005, 40 at the search's unrounded 1.00524): the
# cubic case and the serving stream both take the whole number 1.0.
K3_ALPHA = 1.0
# DRAM bytes (read + write) per launch from the ncu capture summarised in
# profiles/p2p_sym_kernel_tps_262k.md and profiles/m2l_tc_kernel_tps_262k.md, taken on the
# n = 262144 case of this workload at leaf capacity 96 and scaled to the bench size: the
# tensor-core M2L by its tile count (408 tiles there), the near field by the point count.
M2L_DRAM_BYTES_PER_TILE = (21.455872e6 + 7424) / 408
P2P_DRAM_BYTES_PER_POINT = (6.971136e6 + 768) / 262144
# the float-float near field (precision 4): profiles/p2p_sym_ff_kernel_tps_262k.md
P2P_FF_DRAM_BYTES_PER_POINT = (6.929152e6 + 512) / 262144


def workload_config(args, n, m_t, fmm_order, world):
    """The `config` object of both arms' JSON lines."""
    return {"workload": WORKLOAD, "n": n, "targets": m_t, "k": 2, "poly_degree": 1, "vecchia_m": 30,
            "nu": NU, "alpha_normalised": ALPHA,
            "ordering": ["random", "maxmin", "hierarchical maximin", "approximate maximin"][args.ordering],
            "leaf_cap": args.leaf_cap, "fmm_order": fmm_order, "precision_mode": args.precision, "tol": 1e-8,
            "parallelism": f"replicas{world}", "l2": "flushed (256 MB write) between timed steps"}


def default_fmm_order(eps=1e-11):
    """The library's order for fmm_order <= 0: ceil(log eps / log 0.55), clamped to 4..60."""
    import math
    return max(4, min(60, math.ceil(math.log(eps) / math.log(0.55))))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--n", type=int, default=None, help="override the point count (smaller parity runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the other arithmetic beside the line (FP64 beside --precision 4, "
                         "precision 4 beside FP64)")
    ap.add_argument("--leaf-cap", type=int, default=96,
                    help="quadtree leaf capacity (96 measured best on this workload: 48 / 64 / 80 / 96 / "
                         "112 gave 0.429 / 0.344 / 0.327 / 0.323 / 0.331 s per solve)")
    ap.add_argument("--ordering", type=int, default=3, choices=[0, 1, 2, 3],
                    help="Vecchia enumeration: 0 random, 1 exact maxmin, 2 hierarchical maximin, "
                         "3 dyadic approximate maximin")
    ap.add_argument("--requests", type=int, default=120, help="serving case: number of requests")
    ap.add_argument("--rates", default="4,16,saturate",
                    help="serving case: Poisson arrival rates (requests/s), comma separated; 'saturate' = all at once")
    ap.add_argument("--max-active", type=int, default=32, help="serving case: jobs in flight")
    ap.add_argument("--sweep-requests", type=int, default=0,
                    help="serving case: requests per Poisson rate below saturation (0: all)")
    ap.add_argument("--n-max", type=int, default=500_000, help="serving case: largest request")
    ap.add_argument("--jobs", type=int, default=64, help="batch case: number of jobs")
    ap.add_argument("--case", default="step", choices=["step", "plan", "matvec", "precond", "cubic", "serving",
                                                       "batch", "tune"],
                    help="step: the bench (plan + fit + evaluation, the JSON contract line); plan / "
                         "matvec / precond: one piece of it repeated --steps times on one plan, for "
                         "profiling; cubic: the cubic-PHS workload (n = 100,000 from 20 clusters, "
                         "k = 3, m = 20, alpha K3_ALPHA, tol 1e-8) timed like a step; serving: the "
                         "serving engine on a stream of requests with Poisson arrivals (n log-uniform in "
                         "[1000, --n-max], k in 1..3) against the same stream served one job at a time "
                         "(each of these prints its own short line); tune: phs_tune_alpha on the bench "
                         "workload (all points) for nu = 1 and nu = 1.5 from the library's default alpha, "
                         "then a fit at the alpha found")
    return ap.parse_args()


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
        "fallback"


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        import statistics
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle leg
def oracle_step(points, f, targets, n_sample, seed=0):
    """The oracle as it stands on a bounded random subsample: normalisation,
    approximate maximin order, brute-force neighbours, Vecchia factor, dense-matvec PCG to 1e-8, dense
    evaluation at the targets.  Returns (seconds, n_sample, iterations)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(f), n_sample, replace=False))
    p, fs = points[idx], f[idx]
    t0 = time.perf_counter()
    xn, c, rho = oracle.normalize(p, 0.25)
    order, _, _ = oracle.amaxmin_order(xn)
    nbr = oracle.knn_prev(xn, order, 30)
    d, o, _ = oracle.vecchia_factor(xn, order, nbr, 30, NU, ALPHA)
    w, beta, it, _ = oracle.pcg(xn, fs, 2, 1, (nbr, d, o), tol=1e-8, maxiter=300)
    yn = (targets - c) * rho
    oracle.interpolant(xn, w, beta, 2, 1, yn)
    return time.perf_counter() - t0, n_sample, it


# One procedure for both CPU legs (the native line's cpu_baseline and the reference arm):
# the oracle on a fixed-size random subsample, its time scaled to the full n by the
# O(n^2) cost of its dense matvec and labelled as an extrapolation.
CPU_SAMPLE = 16384


def cpu_record(measured, iters, n_full, repeats):
    """The JSON object describing the extrapolated oracle time (both CPU legs)."""
    scale = (n_full / CPU_SAMPLE) ** 2
    return {"value": measured * scale, "unit": "s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"oracle fit (approximate maximin order, brute-force neighbours, Vecchia m=30, dense-matvec "
                      f"PCG to 1e-8, {iters} iters, dense evaluation at 1000 targets) on a {CPU_SAMPLE}-point random "
                      f"subsample of {WORKLOAD}; mean of {repeats} runs {measured:.2f} s, extrapolated by "
                      f"(n/{CPU_SAMPLE})^2 to n={n_full}",
            "measured_s": measured, "n_sample": CPU_SAMPLE, "repeats": repeats, "extrapolated": True}


def cpu_baseline(points, f, targets, n_full, repeats=2):
    runs = [oracle_step(points, f, targets[:1000], CPU_SAMPLE, seed=i) for i in range(repeats)]
    return cpu_record(sum(r[0] for r in runs) / repeats, runs[-1][2], n_full, repeats)


# --------------------------------------------------------------------------- serving
def serve_stream(phs, reqs, arrivals, max_active, threads=4):
    """Submit the requests at their arrival times (s from the start) to a server with
    max_active slots; returns per-request latencies and the server's statistics."""
    sv = phs.Server(max_active=max_active, setup_threads=threads)
    t0 = time.perf_counter()
    ids = []
    for r, ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        o = phs.options(r["k"], alpha=K3_ALPHA) if r["k"] == 3 else phs.options(r["k"])
        ids.append(sv.submit(r["points"], r["f"], r["targets"], r["k"], vecchia_m=30, opts=o))
    res = [sv.wait(i, allow_not_converged=True) for i in ids]
    st = sv.stats()
    sv.close()
    times = [r[4] for r in res]
    lat = sorted(t[3] - t[0] for t in times)
    span = max(t[3] for t in times) - min(t[0] for t in times)
    import numpy as np
    return {"_service_s": [t[3] - t[1] for t in times],
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "solves_per_s": len(reqs) / span, "span_s": span,
            "converged": int(sum(r[3]["converged"] for r in res)),
            "max_true_rel_res": float(max(r[3]["rel_res_true"] for r in res)),
            "max_concurrent": st["max_concurrent"], "ticks": st["ticks"],
            "mean_jobs_per_tick": st["job_iterations"] / max(st["ticks"], 1),
            "not_converged": [{"n": len(q["f"]), "k": q["k"], "iters": r[3]["iters"],
                               "rel_res_true": r[3]["rel_res_true"]}
                              for q, r in zip(reqs, res) if not r[3]["converged"]]}


def batch_case(args, phs):
    """Config-4 style batch: k = 4 / 5 jobs (Franke function, n log-uniform in [2000,
    200000], Sobol points as in Sec. 3.3) at tol 1e-8 in precision 4 (float-float inside
    FP64 refinement for k = 4, the FP64 operator for k = 5) and autotuned leaf capacity,
    all submitted at once to the engine (one tick advances every active job), against
    the same jobs one at a time."""
    import numpy as np

    import synth
    jobs = synth.batch_jobs(args.jobs)
    out = {"case": "batch", "metric": "jobs/s for a batch of k = 4/5 interpolation jobs to 1e-8",
           "jobs": len(jobs), "points_total": int(sum(len(j["f"]) for j in jobs)),
           "k_mix": {str(k): sum(j["k"] == k for j in jobs) for k in (4, 5)}, "vecchia_m": 50, "precision": 4}

    def run(max_active, subset=None):
        js = jobs if subset is None else subset
        sv = phs.Server(max_active=max_active, setup_threads=8)
        t0 = time.perf_counter()
        ids = [sv.submit(j["points"], j["f"], j["targets"], j["k"], vecchia_m=50,
                         opts=phs.options(j["k"], precision=4, leaf_cap=0)) for j in js]
        res = [sv.wait(i, allow_not_converged=True) for i in ids]
        dt = time.perf_counter() - t0
        st = sv.stats()
        sv.close()
        return {"wall_s": dt, "jobs_per_s": len(js) / dt, "converged": int(sum(r[3]["converged"] for r in res)),
                "max_true_rel_res": float(max(r[3]["rel_res_true"] for r in res)),
                "iters_mean": float(np.mean([r[3]["iters"] for r in res])),
                "max_concurrent": st["max_concurrent"], "ticks": st["ticks"],
                "mean_jobs_per_tick": st["job_iterations"] / max(st["ticks"], 1),
                "by_k": {str(k): {"converged": sum(1 for j, r in zip(js, res) if j["k"] == k and r[3]["converged"]),
                                  "jobs": sum(1 for j in js if j["k"] == k),
                                  "largest_n_converged": max([len(j["f"]) for j, r in zip(js, res)
                                                              if j["k"] == k and r[3]["converged"]], default=0),
                                  "smallest_n_not_converged": min([len(j["f"]) for j, r in zip(js, res)
                                                                   if j["k"] == k and not r[3]["converged"]],
                                                                  default=0)}
                         for k in (4, 5)}}

    # warm-up: one job per (k, floor(log2 n)) fills the leaf-capacity tuner and the
    # operator caches that the timed runs then share
    seen, warm = set(), []
    for j in jobs:
        key = (j["k"], int(np.log2(len(j["f"]))))
        if key not in seen:
            seen.add(key)
            warm.append(j)
    run(8, warm)
    out["batched"] = run(min(64, len(jobs)))
    out["sequential"] = run(1)
    print(json.dumps(out))


def fifo_latencies(arrivals, service):
    """Latencies of requests served one at a time in arrival order (a single FIFO
    server): request i starts at max(a_i, end of request i-1) and ends s_i later; its
    latency is end_i - a_i.  Arrivals must be non-decreasing."""
    import numpy as np

    done, lat = 0.0, []
    for a_, s_ in zip(arrivals, service):
        done = max(float(a_), done) + float(s_)
        lat.append(done - float(a_))
    return np.asarray(lat)


def serving_case(args, phs):
    import numpy as np

    import synth
    reqs = synth.serving_requests(args.requests, n_hi=args.n_max)
    out = {"case": "serving", "metric": "serving p50/p99 latency and solves/s at 1e-8 (FP64)",
           "requests": len(reqs), "n_range": [1000, args.n_max],
           "points_total": int(sum(len(r["f"]) for r in reqs)),
           "k_mix": {str(k): sum(r["k"] == k for r in reqs) for k in (1, 2, 3)},
           "max_active": args.max_active,
           "alpha_by_k": {str(k): (K3_ALPHA if k == 3 else phs.options(k).alpha) for k in (1, 2, 3)}, "rates": {}}
    # Sequential arm: one job at a time (max_active = 1 admits the next job only when the
    # last is done), so under any arrival times its latencies follow from each job's own
    # service time by the FIFO single-server recursion start_i = max(a_i, done_{i-1}).  It
    # runs live once (all requests submitted at once); the other rates use the recursion
    # on those measured service times, marked "simulated".  The batched arm runs live at
    # every rate, on the first --sweep-requests requests below saturation.
    seq = serve_stream(phs, reqs, np.zeros(len(reqs)), 1)
    svc = seq.pop("_service_s")

    def fifo(arr, svc_):
        lat = fifo_latencies(arr, svc_)
        done = float(arr[-1]) + float(lat[-1])
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "solves_per_s": len(arr) / (done - float(np.min(arr))),
                "simulated": True}

    for rate in args.rates.split(","):
        if rate == "saturate":
            b = serve_stream(phs, reqs, np.zeros(len(reqs)), args.max_active)
            b.pop("_service_s")
            out["rates"][rate] = {"requests": len(reqs), "batched": b, "sequential": seq}
        else:
            ns = min(len(reqs), args.sweep_requests) if args.sweep_requests > 0 else len(reqs)
            arr = synth.poisson_arrivals(ns, float(rate))
            b = serve_stream(phs, reqs[:ns], arr, args.max_active)
            b.pop("_service_s")
            out["rates"][rate] = {"requests": ns, "batched": b, "sequential": fifo(arr, svc[:ns])}
    out["sequential_note"] = ("sequential latencies at the Poisson rates come from the FIFO recursion over the "
                              "service times measured live in the all-at-once sequential run")
    print(json.dumps(out))


# --------------------------------------------------------------------------- native leg
def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    import numpy as np

    import synth

    wl = synth.workload(WORKLOAD, n=args.n)
    points, f, targets = wl["points"], wl["f"], wl["targets"]
    n, m_t = len(f), len(targets)

    if args.impl == "reference":
        if rank != 0:
            return
        dts, it = [], 0
        for i in range(args.warmup + args.steps):
            dt, _, it = oracle_step(points, f, targets[:1000], CPU_SAMPLE, seed=i)
            if i >= args.warmup:
                dts.append(dt)
        measured = float(np.mean(dts))
        cb = cpu_record(measured, it, n, args.steps)
        v = cb["value"]
        # value: the full-size time by the shared extrapolation (the metric is defined at n);
        # ms_per_step: what one timed step actually took (the sampled oracle fit)
        print(json.dumps({"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": measured * 1e3, "value_extrapolated": True,
                          "higher_is_better": False,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "impl": "reference", "config": workload_config(args, n, m_t, default_fmm_order(), 1),
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_2608_11462_b300 as phs

    L = phs.lib()
    opts = phs.options(2, precision=args.precision, tol=1e-8, nu=NU, alpha=ALPHA, leaf_cap=args.leaf_cap,
                       ordering=args.ordering)
    pts_d = torch.tensor(points, device=dev)
    f_d = torch.tensor(f, device=dev)
    tg_d = torch.tensor(targets, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.case == "cubic":
        wc = synth.workload("cubic_mix")
        pc, fc, tc = (torch.tensor(wc[key], device=dev) for key in ("points", "f", "targets"))
        copts = phs.options(3, tol=1e-8, maxiter=400, precision=args.precision, alpha=K3_ALPHA)
        res = []
        # the timed steps run as a user would (near field beside the far field); one more
        # step with phase timing (near field serialised) gives the breakdown
        for i in range(args.warmup + args.steps + 1):
            timing = i == args.warmup + args.steps
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan = phs.Plan(pc, 3, vecchia_m=20, opts=copts)
            plan.set_timing(timing)
            w, beta, info = plan.fit(fc)
            plan.eval(w, beta, tc)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tim = plan.timing() if timing else None
            plan.close()
            if timing:
                phase_tim = tim
            elif i >= args.warmup:
                res.append((e0.elapsed_time(e1) / 1e3, info))
        if rank == 0:
            t = float(np.mean([r[0] for r in res]))
            info = res[-1][1]
            print(json.dumps({"case": "cubic", "workload": "cubic_mix", "n": len(wc["f"]), "k": 3, "vecchia_m": 20,
                              "alpha": K3_ALPHA,
                              "precision": args.precision, "value_s": t, "steps": args.steps, "iters": info["iters"],
                              "rel_res_true": info["rel_res_true"], "ms_plan": info["ms_plan"],
                              "ms_fit": info["ms_fit"], "ms_matvec_avg": info["ms_matvec_avg"],
                              "phases_ms_per_call": {k_: (v[0] / v[1] if v[1] else 0.0)
                                                     for k_, v in phase_tim.items()},
                              "phases_note": "one extra step with phase timing (near field serialised)"}))
        return
    if args.case == "serving":
        if rank == 0:
            serving_case(args, phs)
        return
    if args.case == "batch":
        if rank == 0:
            batch_case(args, phs)
        return
    if args.case == "tune":
        if rank == 0:
            # the search runs on another draw of the same recipe, the fits on the bench's own
            held = synth.workload(WORKLOAD, n=n, seed=TUNE_SEED)
            hp, hf = torch.tensor(held["points"], device=dev), torch.tensor(held["f"], device=dev)
            out = {"case": "tune", "workload": WORKLOAD, "n": n, "vecchia_m": 30, "tol": 1e-8,
                   "search_on": f"{WORKLOAD} drawn with seed {TUNE_SEED}", "runs": []}
            for nu in (NU, 1.5):
                o = phs.options(2, tol=1e-8, nu=nu, leaf_cap=args.leaf_cap, ordering=args.ordering, maxiter=200)
                a0 = o.alpha
                t0 = time.perf_counter()
                a, it_tune = phs.phs_tune_alpha(hp, hf, 2, vecchia_m=30, opts=o, n_sample=n)
                t_tune = time.perf_counter() - t0
                run = {"nu": nu, "alpha_start": a0, "alpha": a, "iters_in_search": it_tune, "s_search": t_tune}
                for tag, al in (("at_alpha", a), ("at_default", a0), ("at_bench_alpha", ALPHA)):
                    o2 = phs.options(2, tol=1e-8, nu=nu, alpha=al, leaf_cap=args.leaf_cap, ordering=args.ordering,
                                     maxiter=200)
                    plan = phs.Plan(pts_d, 2, fmm_order=0, vecchia_m=30, opts=o2)
                    try:
                        _, _, info = plan.fit(f_d)
                        run[tag] = {"alpha": al, "iters": info["iters"], "rel_res_true": info["rel_res_true"]}
                    except phs.PhsError as e:
                        run[tag] = {"alpha": al, "error": str(e)}
                    plan.close()
                out["runs"].append(run)
            print(json.dumps(out))
        return
    if args.case != "step":
        # one piece of the step on the bench workload, for profilers; no timing contract
        reps = max(1, args.steps)
        if args.case == "plan":
            for _ in range(reps):
                phs.Plan(pts_d, 2, fmm_order=0, vecchia_m=30, opts=opts).close()
        else:
            p = phs.Plan(pts_d, 2, fmm_order=0, vecchia_m=30, opts=opts)
            for _ in range(reps):
                p.matvec(f_d) if args.case == "matvec" else p.precond(f_d)
            torch.cuda.synchronize(dev)
            p.close()
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"case": args.case, "n": n, "repeats": reps, "workload": WORKLOAD}))
        return
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(timing=False):
        plan = phs.Plan(pts_d, 2, fmm_order=0, vecchia_m=30, opts=opts)
        if timing:
            plan.set_timing(True)
        w, beta, info = plan.fit(f_d)
        pred = plan.eval(w, beta, tg_d)
        tim = plan.timing() if timing else None
        work = plan.work()
        kw = plan.kernel_work()
        sizes = plan.frame()[1]
        plan.close()
        return info, tim, (work, kw), sizes, pred

    for _ in range(args.warmup):
        step()
    times, infos, tims = [], [], []
    clocks = ClockSampler(local)
    launches0 = L.phs_kernel_launches()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info, _, (work, kwork), sizes, pred = step(timing=False)
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1) / 1e3)
        infos.append(info)
    clk = clocks.stop()
    launches = (L.phs_kernel_launches() - launches0) // args.steps
    # phase breakdown from separate steps with the library's phase timing on (events around
    # each phase; the near field then stays on the main stream instead of overlapping the
    # far field), outside the timed region
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        barrier()
        _, tim, _, _, _ = step(timing=True)
        tims.append(tim)
    t_step = float(np.mean(times))
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_step], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())

    # ---- the other arithmetic on the same workload: beside a precision-4 line the plain
    # FP64 solve, beside the FP64 line the precision-4 solve (float-float bulk inside FP64
    # refinement; its true residual is checked with the FP64 operator).  Untimed steps
    # for the headline; each timed with events like a step, the first of three dropped.
    def other_solve(prec):
        oo = phs.options(2, precision=prec, tol=1e-8, nu=NU, alpha=ALPHA, leaf_cap=args.leaf_cap,
                         ordering=args.ordering)
        ts, inf = [], None
        for i in range(3):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            po = phs.Plan(pts_d, 2, fmm_order=0, vecchia_m=30, opts=oo)
            wo, bo, inf = po.fit(f_d)
            po.eval(wo, bo, tg_d)
            e1.record(stream)
            barrier()
            po.close()
            if i > 0:
                ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.mean(ts)), inf

    fp64_cmp = None
    if args.precision != 0 and not args.no_fp64_compare:
        t64, i64 = other_solve(0)
        fp64_cmp = {"fp64_step_s": t64, "fp64_iters": i64["iters"], "fp64_rel_res_true": i64["rel_res_true"],
                    "speedup_vs_fp64": t64 / t_step}
    elif args.precision == 0 and not args.no_fp64_compare:
        t4, i4 = other_solve(4)
        fp64_cmp = {"precision4_step_s": t4, "precision4_iters": i4["iters"],
                    "precision4_outer_iters": i4["outer_iters"], "precision4_rel_res_true": i4["rel_res_true"],
                    "precision4_speedup": t_step / t4}

    # ---- end to end from host buffers through the C ABI
    e2e_times = []
    for i in range(max(1, min(args.steps, 2))):
        barrier()
        t0 = time.perf_counter()
        phs.phs_fit_predict_host(points, f, targets, 2, vecchia_m=30, opts=opts)
        torch.cuda.synchronize(dev)
        e2e_times.append(time.perf_counter() - t0)
    e2e = float(np.mean(e2e_times))
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([e2e], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = float(tt.item())

    # ---- roofline of the dominant kernel (per-launch algorithmic work / event-timed duration)
    peaks, peak_kind = load_peaks()
    agg = {}
    for tim in tims:
        for k_, (ms, calls) in tim.items():
            a = agg.setdefault(k_, [0.0, 0])
            a[0] += ms
            a[1] += calls
    phases = {k_: v for k_, v in agg.items() if k_ in ("p2p", "m2l", "upward", "downward", "precond", "vector")}
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2032.0))
    ms_p2p = phases["p2p"][0] / max(phases["p2p"][1], 1)
    if args.precision == 4:
        # float-float near field (nearfield_ff.cu): FP32-pipe operations per pair as written
        # there -- coordinates 16, s = r^2 19, logarithm 32, s log s 4, row term and sum 12 --
        # 83 per pair, plus 12 where the pair also feeds a column sum
        fp32_peak_g = 148 * 128 * sm_mhz_max * 1e6 / 1e9
        p2p_ops = 83 * kwork["p2p_pairs"] + 12 * kwork["p2p_column_pairs"]
        ach = p2p_ops / (ms_p2p / 1e3) / 1e9
        roof_p2p = {"kernel": "p2p_sym_ff_kernel<2> + p2p_gather", "bound": "alu", "achieved": ach,
                    "peak": fp32_peak_g, "unit": "G FP32-pipe instr/s", "frac": ach / fp32_peak_g,
                    "peak_source": f"derived: 148 SMs x 128 FP32 lanes x {sm_mhz_max:.0f} MHz",
                    "work_per_launch": f"{kwork['p2p_pairs']} pairs evaluated ({kwork['p2p_column_pairs']} with "
                                       f"column sums) = {p2p_ops} FP32-pipe instr; {work['near_pairs']} ordered near "
                                       f"pairs", "ms_per_launch": ms_p2p,
                    "gpairs_per_s": work["near_pairs"] / (ms_p2p / 1e3) / 1e9,
                    "traffic": P2P_FF_DRAM_BYTES_PER_POINT * n
                    if P2P_FF_DRAM_BYTES_PER_POINT else None}
    else:
        # FP64 pipe: 2 instructions (DFMA, DMUL or DADD) per clock per SM.  Per evaluated pair:
        # DADD + 2 DFMA (r^2 = a_i + a_j - 2 x_i.x_j), 4 DFMA + DADD (table log), DMUL
        # (r^2 log r^2), DFMA (row sum) = 10; one more DFMA where the pair also feeds a column sum
        fp64_peak_g = 148 * 2 * sm_mhz_max * 1e6 / 1e9
        p2p_ops = 10 * kwork["p2p_pairs"] + kwork["p2p_column_pairs"]
        ach = p2p_ops / (ms_p2p / 1e3) / 1e9
        roof_p2p = {"kernel": "p2p_sym_kernel<2> + p2p_gather", "bound": "alu", "achieved": ach,
                    "peak": fp64_peak_g, "unit": "G FP64-pipe instr/s", "frac": ach / fp64_peak_g,
                    "peak_source": f"derived: 148 SMs x 2 FP64 instr/clk x {sm_mhz_max:.0f} MHz",
                    "work_per_launch": f"{kwork['p2p_pairs']} pairs evaluated ({kwork['p2p_column_pairs']} with "
                                       f"column sums) = {p2p_ops} FP64 instr; {work['near_pairs']} ordered near pairs",
                    "ms_per_launch": ms_p2p, "gpairs_per_s": work["near_pairs"] / (ms_p2p / 1e3) / 1e9,
                    "traffic": P2P_DRAM_BYTES_PER_POINT * n}
    ms_m2l = phases["m2l"][0] / max(phases["m2l"][1], 1)
    roof_m2l = None
    if kwork["tc_steps"] > 0:
        flops = 2.0 * kwork["tc_steps"] * kwork["tc_mmas_per_step"] * kwork["tc_mma_macs"]
        pk = float(peaks.get("bf16_tflops_sustained", 1371.7))
        ach = flops / (ms_m2l / 1e3) / 1e12
        roof_m2l = {"kernel": "m2l_tc_kernel<4>", "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                    "frac": ach / pk, "peak_source": "measured bf16 (sustained, kernel inside a long step)",
                    "work_per_launch": f"{kwork['tc_steps']} steps x {kwork['tc_mmas_per_step']} digit-plane "
                                       f"products x {kwork['tc_mma_macs']} MAC (bf16, FP32 accumulate; issued as "
                                       f"tcgen05.mma spanning up to 256 output columns)",
                    "ms_per_launch": ms_m2l,
                    "traffic": M2L_DRAM_BYTES_PER_TILE * kwork["tc_tiles"]}
    if roof_m2l is not None and ms_m2l > ms_p2p:
        roof, roof_other = roof_m2l, {"roofline_p2p": roof_p2p}
    else:
        roof, roof_other = roof_p2p, ({"roofline_m2l": roof_m2l} if roof_m2l else {})
    roof["peak_kind"] = peak_kind
    # the preconditioner apply (HBM-bound) alongside: 2 passes over the factor + vectors
    pre_ms = phases["precond"][0] / max(phases["precond"][1], 1)
    nnz = n * 31
    pre_bytes = 2 * nnz * 12 + 4 * n * 8
    pre = {"bound": "hbm", "achieved": pre_bytes / (pre_ms / 1e3) / 1e9, "peak": float(peaks["hbm_gbs"]),
           "unit": "GB/s", "ms_per_launch": pre_ms, "bytes_per_launch": pre_bytes}
    pre["frac"] = pre["achieved"] / pre["peak"]

    # FMM throughput (n / t(matvec)): every density of the Hadamard form, the whole FP64
    # matvec (near field + far field), timed with events inside the fit
    mv_ms = float(np.mean([inf["ms_matvec_avg"] for inf in infos]))
    fmm = {"ms_per_matvec": mv_ms, "applies_per_s": 1e3 / mv_ms, "gpts_per_s": n / (mv_ms / 1e3) / 1e9,
           "densities": int(sizes[4])}
    if roof_m2l is not None:
        # the method's work: one complex P x P translation per V-list entry and density,
        # 8 P^2 real flops (P = p + 1 coefficients), against the digit-plane MMA work above
        P = int(sizes[3]) + 1
        meth = 8.0 * P * P * int(sizes[4]) * work["m2l_translations"]
        roof_m2l["method_flops_per_launch"] = meth
        roof_m2l["method_tflops"] = meth / (ms_m2l / 1e3) / 1e12
        roof_m2l["v_list_entries"] = work["m2l_translations"]
        roof_m2l["mma_flops_per_method_flop"] = 2.0 * kwork["tc_steps"] * kwork["tc_mmas_per_step"] * \
            kwork["tc_mma_macs"] / meth

    info = infos[-1]
    out = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f64", 4: "f64+ff32"}.get(args.precision, "f64+f32"), "data": "synthetic",
        "fits_per_s": world / t_step,
        "config": workload_config(args, n, m_t, int(sizes[3]), world),
        "pcg": {"iters": info["iters"], "outer_iters": info["outer_iters"], "converged": info["converged"],
                "rel_res_true": info["rel_res_true"], "ms_plan": info["ms_plan"], "ms_fit": info["ms_fit"],
                "ms_matvec_avg": info["ms_matvec_avg"]},
        "phases_ms_per_step": {k_: v[0] / len(tims) for k_, v in agg.items()},
        "phases_note": f"from {len(tims)} further steps with the library's phase timing on, outside the timed "
                       "region: it keeps the near field on the plan's stream (the timed steps overlap it with the "
                       "upward pass and M2L on a second stream), so each phase's events time that phase alone",
        **({("fp64_comparison" if args.precision != 0 else "precision4_comparison"): fp64_cmp} if fp64_cmp else {}),
        "fmm_throughput": fmm,
        "roofline": roof, **roof_other, "roofline_precond": pre, "clocks": clk, "gpu_launches": int(launches),
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(16 * n + 8 * n + 16 * m_t),
                "d2h_bytes_per_step": int(8 * n + 8 * 3 + 8 * m_t)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(points, f, targets, n)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
