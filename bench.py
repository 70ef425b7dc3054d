"""Benchmark: the serving stream of Dual (O-)BDRS solves on one B300 (or N replicas).

Workload (one "step"): a seeded stream of ``--requests`` OT solves with Poisson arrivals at
``--rate`` requests/s, grid sizes drawn 50% 32x32, 35% 64x64, 15% 128x128, histogram classes drawn
per request (uniform-random, 1-5 component Gaussian mixtures, Cauchy-like, 90%-sparse floored at
1e-15), eps0 = 1, lambda = 1, FP32 exp / FP64 potentials, certificate every ``--cert-every``
iterations, each request stopping at a 1% relative certified gap or ``--max-iters``.

Metric: implicit entries per second over the whole stream (2 n m entries per iteration), with
p50/p99 solve latency (arrival to completion) and time to certified gap beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank serves its own stream (independent replicas, weak scaling);
the reference arm (the FP64 CPU oracle) runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ot_inputs as I  # noqa: E402

METRIC = "implicit entries/s per dual sweep (serving stream); time to certified gap; p50/p99 solve latency"
UNIT = "entries/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--engine", default="batched", choices=["batched", "serial"])
    ap.add_argument("--slots", type=int, default=256, help="server slots (batched engine)")
    ap.add_argument("--serial-steps", type=int, default=1,
                    help="also time this many steps of one-at-a-time solves (same stop rule) for comparison")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=32.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--burst", action="store_true", help="every request arrives at t = 0 (profiling)")
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--cert-every", type=int, default=100)
    ap.add_argument("--tol-rel", type=float, default=0.01)
    ap.add_argument("--lam", type=float, default=1.5, help="arms workload: overrelaxation lambda")
    ap.add_argument("--serve-lam", type=float, default=1.0, help="serve workload: overrelaxation lambda")
    ap.add_argument("--n-points", type=int, default=1 << 16, help="ablation workload: points per cloud")
    ap.add_argument("--eta", type=float, default=0.1, help="ablation and transfer workloads: eps0")
    ap.add_argument("--budget-s", type=float, default=600.0, help="transfer workload: wall-time budget")
    ap.add_argument("--reverse", action="store_true", help="transfer workload: the backward direction")
    ap.add_argument("--instances", type=int, default=8, help="delay workload: instance pairs")
    ap.add_argument("--delay-set", default="clouds", choices=["clouds", "grids"],
                    help="delay workload: 1024-point uniform-weight clouds (exact assignment) or 16x16 grid "
                         "histograms of the four classes (exact transport LP)")
    ap.add_argument("--seed", type=int, default=2609)
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--workload", default="serve",
                    choices=["serve", "sweep", "project", "arms", "ablation", "delay", "load", "transfer",
                             "precision"],
                    help="serve: the serving stream (the bench line); sweep: one resident instance, "
                         "fast iterations only (kernel roofline and profiling)")
    ap.add_argument("--size", type=int, default=512, help="sweep workload: s for an s x s grid, or -n for "
                                                          "n RGB points")
    ap.add_argument("--iters", type=int, default=10, help="sweep workload: iterations per step")
    ap.add_argument("--precision", default="mufu", choices=["mufu", "comp", "fp64"])
    ap.add_argument("--skip", type=int, default=0, help="sweep workload: untimed iterations before the warm-up")
    ap.add_argument("--refine-on", type=float, default=0.0,
                    help="sweep workload: refine_on of the fast sweeps (0: off)")
    ap.add_argument("--ttg-refine-on", type=float, default=2.0 ** -6,
                    help="time-to-gap leg: refine_on of the fast sweeps (0: off)")
    ap.add_argument("--ttg-requests", type=int, default=64,
                    help="time-to-gap leg: requests of the stream solved under the stop rule with --ttg-max-iters")
    ap.add_argument("--ttg-max-iters", type=int, default=100000)
    ap.add_argument("--cmp-n", type=int, default=4,
                    help="time-to-gap leg: 64x64 requests also solved with the compensated exponent")
    ap.add_argument("--no-legs", action="store_true", help="skip the time-to-gap and config-1 legs")
    ap.add_argument("--study-n", type=int, default=6, help="precision workload: requests rerun per arm")
    ap.add_argument("--study-base", default="0:0",
                    help="precision workload: refine_on:refine_tol of the first pass over the stream")
    ap.add_argument("--study-arms", default="comp,centred",
                    help="precision workload: arms rerun on the sample (comp, centred, mufu; @ON:TOL sets the "
                         "fast sweeps' refinement thresholds)")
    return ap.parse_args()


# ----------------------------------------------------------------------------------------------
# clocks during the timed region (nvidia-smi sampling)
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------------------------
def combine_over_ranks(td, device, t_step, entries, e2e_t, e2e_entries):
    """Whole-job numbers from per-rank ones: the slowest rank's time, the sum of the work.

    Every rank serves its own stream (independent replicas), so the only exchange is this one."""
    import torch
    tt = torch.tensor([t_step, entries, e2e_t, e2e_entries], dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(tt) for _ in range(td.get_world_size())]
    td.all_gather(gathered, tt)
    return (max(float(g[0]) for g in gathered), sum(float(g[1]) for g in gathered),
            max(float(g[2]) for g in gathered), sum(float(g[3]) for g in gathered))


FAST_DRAM_BYTES_PER_ENTRY = (0.454266368e9 + 1.922718e9) / 4.52e11


def make_stream(args, rank: int):
    reqs = I.serving_stream(args.requests, args.seed + 7919 * rank, args.rate)
    if args.burst:
        for r in reqs:
            r.arrival_s = 0.0
    probs = [I.request_problem(r) for r in reqs]
    return reqs, probs


def solve_params(args):
    return dict(eps0=1.0, lam=args.serve_lam, max_iters=args.max_iters, cert_every=args.cert_every, precision="mufu",
                tol_rel=args.tol_rel)


def run_serial(ctx, reqs, probs, dev_inputs, args, host: bool):
    """One-at-a-time FIFO serving: each request starts at max(arrival, previous completion)."""
    import torch
    t0 = time.perf_counter()
    lat, ttg, entries, conv, ttg_conv = [], [], 0.0, 0, []
    h2d = d2h = 0
    for r, p, dv in zip(reqs, probs, dev_inputs):
        now = time.perf_counter() - t0
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        ts = time.perf_counter()
        if host:
            f, g, res = ctx.solve(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                                  **solve_params(args))
            h2d += p.x.nbytes + p.y.nbytes + p.a.nbytes + p.b.nbytes
            d2h += f.nbytes + g.nbytes
        else:
            x, y, a, b = dv
            f, g, res = ctx.solve(x, y, a, b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                                  **solve_params(args))
        te = time.perf_counter()
        lat.append(te - t0 - r.arrival_s)
        ttg.append(te - ts)
        entries += 2.0 * p.n * p.m * res["iters"]
        conv += res["stop"] == "tol"
        if res["stop"] == "tol":
            ttg_conv.append(te - ts)
    return dict(latency=lat, ttg=ttg, entries=entries, converged=conv, h2d=h2d, d2h=d2h, ttg_conv=ttg_conv)


def run_batched(srv, reqs, probs, dev_inputs, args, host: bool):
    """Continuous batching: requests are submitted at their arrival times to the server, which
    admits them at certificate boundaries and batches all running solves in each launch."""
    t0 = time.perf_counter()
    ids = []
    h2d = d2h = 0
    for r, p, dv in zip(reqs, probs, dev_inputs):
        now = time.perf_counter() - t0
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        if host:
            ids.append(srv.submit(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                                  **solve_params(args)))
            h2d += p.x.nbytes + p.y.nbytes + p.a.nbytes + p.b.nbytes
        else:
            x, y, a, b = dv
            ids.append(srv.submit(x, y, a, b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                                  **solve_params(args)))
    lat, ttg, entries, conv, ttg_conv = [], [], 0.0, 0, []
    for rid, p in zip(ids, probs):
        f, g, res = srv.wait(rid, -1.0)
        d2h += f.nbytes + g.nbytes
        lat.append(res["latency_s"])
        ttg.append(res["latency_s"] - res["queue_s"])
        entries += 2.0 * p.n * p.m * res["iters"]
        conv += res["stop"] == "tol"
        if res["stop"] == "tol":
            ttg_conv.append(res["latency_s"] - res["queue_s"])
    return dict(latency=lat, ttg=ttg, entries=entries, converged=conv, h2d=h2d, d2h=d2h, ttg_conv=ttg_conv)


def flush_l2(buf):
    buf.add_(1.0)


# ----------------------------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------------------------
def _oracle_requests(task):
    """One host process of the CPU baseline: the oracle as it stands (dense FP64 numpy) on its share
    of the stream's requests, in arrival order, each for up to max_iters iterations with its
    certificates and stop rule, until budget_s seconds have passed.  Returns (entries, seconds,
    [n:iterations])."""
    reqs, max_iters, cert_every, tol_rel, budget_s, max_n = task
    import oracle as O
    t0 = time.perf_counter()
    entries = 0.0
    done = []
    for r in reqs:
        p = I.request_problem(r)
        if p.n > max_n:
            continue
        C = O.cost_matrix(p.x, p.y, p.kappa)
        a = np.maximum(p.a, 1e-15)
        a = a / a.sum()
        b = np.maximum(p.b, 1e-15)
        b = b / b.sum()
        st = O.DualState.initial(p.n, p.m)
        la, lb = np.log(a), np.log(b)
        k = 0
        while k < max_iters:
            st = O.dual_obdrs_step(st, la, lb, C, 1.0, 1.0)
            k += 1
            entries += 2.0 * p.n * p.m
            if cert_every > 0 and k % cert_every == 0:
                cert = O.certificate_of(st, a, b, C, p.omega)
                if (cert["U"] - cert["L"]) <= tol_rel * abs(cert["U"]):
                    break
            if time.perf_counter() - t0 > budget_s:
                break
        done.append(f"{p.n}:{k}")
        del C
        if time.perf_counter() - t0 > budget_s:
            break
    return entries, time.perf_counter() - t0, done


class OraclePool:
    """The CPU baseline's host processes: one single-threaded oracle process per host core (spawned,
    so that no child inherits the parent's CUDA state).  The stream's requests are independent, so
    request i goes to process i mod W; the oracle's arithmetic is unchanged.  The 128 x 128 class
    (a 2 GB dense cost matrix and about 8 GB of temporaries per process) is included when the host
    has the memory for every process."""

    def __init__(self):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.workers = max(1, os.cpu_count() or 1)
        avail = 0
        try:
            with open("/proc/meminfo") as f:
                for line in f:
                    if line.startswith("MemAvailable:"):
                        avail = int(line.split()[1]) * 1024
        except OSError:
            pass
        self.max_n = 16384 if avail >= self.workers * (12 << 30) else 4096
        self.pool = mp.get_context("spawn").Pool(self.workers)

    def sample(self, args, reqs, budget_s: float):
        tasks = [(reqs[w::self.workers], args.max_iters, args.cert_every, args.tol_rel, budget_s, self.max_n)
                 for w in range(self.workers)]
        t0 = time.perf_counter()
        outs = self.pool.map(_oracle_requests, tasks)
        wall = time.perf_counter() - t0
        entries = sum(o[0] for o in outs)
        done = [d for o in outs for d in o[2]]
        return entries / wall, wall, done

    def describe(self, budget_s: float, done) -> str:
        sizes = {}
        for d in done:
            n = d.split(":")[0]
            sizes[n] = sizes.get(n, 0) + 1
        return (f"oracle (dense FP64 numpy) in {self.workers} spawned single-threaded processes, request i of the "
                f"stream on process i mod {self.workers}, each for ~{budget_s:.0f} s; requests with n <= "
                f"{self.max_n}; requests started per n: {sizes}")

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    reqs, probs = make_stream(args, 0)
    pool = OraclePool()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, done = pool.sample(args, reqs, args.cpu_sample_s)
        if i >= args.warmup:
            vals.append((v, dt, done))
    pool.close()
    v = statistics.median([x[0] for x in vals])
    sample = pool.describe(args.cpu_sample_s, vals[-1][2])
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median([x[1] for x in vals]),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "serving stream, mixed 32x32/64x64/128x128 grid histograms",
                      "requests": args.requests, "rate_per_s": args.rate, "max_iters": args.max_iters,
                      "tol_rel": args.tol_rel, "seed": args.seed},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------
def _oracle_config1(task):
    """The oracle's full config-1 run (32 x 32 grid, eps0 = 1, lambda = 1, 2000 iterations, a
    certificate every 100) in one host process: (seconds, [(k, U, L)], best f, best g)."""
    seed, iters, cert_every = task
    import oracle as O
    prob = I.grid_problem(32, seed)
    t0 = time.perf_counter()
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    ro = O.solve(prob.a, prob.b, C, 1.0, 1.0, iters, cert_every, prob.omega)
    return time.perf_counter() - t0, ro["history"], ro["best"]["f"], ro["best"]["g"]


def run_config1(P, ctx, args, oracle_res):
    """Config 1 on the GPU (FP64 sweeps, and FP32 with compensated certificates) beside the oracle's
    run of the same problem: wall time and the certified bounds at every certificate."""
    import torch
    seed, iters, ce = args.seed, 2000, 100
    prob = I.grid_problem(32, seed)
    out = {"workload": "32x32 grid, uniform-random weights, eps0 = 1, lambda = 1, 2000 iterations, certificate "
                       "every 100", "seed": seed}
    fg = {}
    for prec in ("fp64", "mufu"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=1.0,
                      precision=prec, cert_every=ce)
        hist = []
        for _ in range(iters // ce):
            r = S.step(ce)
            hist.append((int(r["iters"]), r["U"], r["L"]))
        fg[prec] = (S.get(P.OT_F_BEST), S.get(P.OT_G_BEST))
        out[prec] = {"seconds": time.perf_counter() - t0, "U_best": r["U_best"], "L_best": r["L_best"],
                     "gap_rel": r["gap_rel"], "best_iter": int(r["best_iter"]), "certificates": hist}
        S.close()
    o_s, o_hist, o_f, o_g = oracle_res
    out["oracle"] = {"seconds": o_s, "certificates": [(int(k), u, l) for k, u, l in o_hist], "cores": 1}
    scale = max(np.abs(o_f).max(), np.abs(o_g).max())
    out["fp64_vs_oracle"] = {"max_abs_U_L": max(max(abs(a[1] - b[1]), abs(a[2] - b[2]))
                                               for a, b in zip(out["fp64"]["certificates"], o_hist)),
                             "potentials_rel": max(np.abs(fg["fp64"][0] - o_f).max(),
                                                   np.abs(fg["fp64"][1] - o_g).max()) / scale}
    out["fp32_vs_fp64"] = {"max_abs_U_L": max(max(abs(a[1] - b[1]), abs(a[2] - b[2]))
                                             for a, b in zip(out["mufu"]["certificates"], out["fp64"]["certificates"])),
                           "potentials_rel": max(np.abs(fg["mufu"][0] - fg["fp64"][0]).max(),
                                                 np.abs(fg["mufu"][1] - fg["fp64"][1]).max()) / scale}
    return out


def run_time_to_gap(P, ctx, args, stream):
    """Time to a certified relative gap under the config's stop rule (--tol-rel, a certificate every
    --cert-every, --ttg-max-iters cap; App. G.3 best-so-far bounds): the first --ttg-requests requests
    of the serving stream, Poisson arrivals, batched server, device-resident inputs.  The fast sweeps
    refine their dominant terms once the FP32 exponent's rounding bound exceeds --ttg-refine-on
    (ot_params.refine_on).  Then --cmp-n of its 64 x 64 requests again with the compensated exponent on
    every iteration, so that each of those results states its certified gap and iterations beside the
    compensated ones."""
    import copy
    import torch
    a2 = copy.copy(args)
    a2.requests, a2.max_iters, a2.burst = args.ttg_requests, args.ttg_max_iters, False
    reqs, probs = make_stream(a2, 0)
    dev = [tuple(torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)) for p in probs]
    srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=args.slots, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = []
    for r, dv in zip(reqs, dev):
        now = time.perf_counter() - t0
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        ids.append(srv.submit(*dv, cost_scale=probs[len(ids)].kappa, omega=probs[len(ids)].omega,
                              zero_mass_floor=1e-15, **dict(solve_params(a2), refine_on=args.ttg_refine_on)))
    res = [srv.wait(i, -1.0)[2] for i in ids]
    makespan = time.perf_counter() - t0
    srv.close()
    conv = [r for r in res if r["stop"] == "tol"]
    ttg = [r["latency_s"] - r["queue_s"] for r in conv]
    lat = [r["latency_s"] for r in res]
    nc = {}
    for q, r in zip(reqs, res):
        if r["stop"] != "tol":
            key = f"{q.s}x{q.s} {q.cls_a}/{q.cls_b}"
            nc.setdefault(key, []).append(round(r["gap_rel"], 5))
    out = {"requests": len(reqs), "max_iters": a2.max_iters, "tol_rel": args.tol_rel, "cert_every": args.cert_every,
           "lambda": args.serve_lam, "rate_per_s": args.rate, "refine_on": args.ttg_refine_on,
           "makespan_s": makespan,
           "converged_frac": len(conv) / len(res),
           "time_to_gap_p50_s": float(np.percentile(ttg, 50)) if ttg else None,
           "time_to_gap_p99_s": float(np.percentile(ttg, 99)) if ttg else None,
           "iters_to_gap_median": float(np.median([r["iters"] for r in conv])) if conv else None,
           "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
           "not_converged_best_gaps": nc,
           "note": "time to gap = admission to the certificate that met the stop rule, converged requests only; "
                   "latency = arrival to result, all requests (those not converged stop at max_iters)"}
    idx = [i for i, q in enumerate(reqs) if q.s == 64][:args.cmp_n]
    if idx:
        srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=len(idx), stream=stream.cuda_stream)
        cids = [srv.submit(*dev[i], cost_scale=probs[i].kappa, omega=probs[i].omega, zero_mass_floor=1e-15,
                           **dict(solve_params(a2), precision="comp")) for i in idx]
        cres = [srv.wait(c, -1.0)[2] for c in cids]
        srv.close()
        out["fp32_vs_compensated"] = [
            {"s": reqs[i].s, "classes": f"{reqs[i].cls_a}/{reqs[i].cls_b}", "seed": reqs[i].seed,
             "fp32": {"iters": int(res[i]["iters"]), "stop": res[i]["stop"], "gap_rel": res[i]["gap_rel"],
                      "U_best": res[i]["U_best"], "L_best": res[i]["L_best"]},
             "compensated": {"iters": int(c["iters"]), "stop": c["stop"], "gap_rel": c["gap_rel"],
                             "U_best": c["U_best"], "L_best": c["L_best"]},
             "gap_rel_diff": res[i]["gap_rel"] - c["gap_rel"]} for i, c in zip(idx, cres)]
    return out


def peaks_for_roofline(probe, clocks):
    # entries/clk/SM bound: min(FP32 lanes / (d + 2), MUFU ex2 lanes); d = 2 for grid workloads
    fp32 = 128.0
    mufu = 32.0
    per_clk = min(fp32 / 4.0, mufu)
    mhz = clocks.get("sm_max_mhz") or 2032.0
    return per_clk * 148 * mhz * 1e6


def run_ours(args, rank: int, world: int):
    import ctypes
    import torch
    import paper_2609_33814_b300 as P
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    dev = int(os.environ.get("LOCAL_RANK", 0))
    # the CPU baseline's spawned oracle processes (rank 0); the oracle's config-1 run starts now on one
    # of them and overlaps the GPU work
    pool = OraclePool() if rank == 0 else None
    c1_async = pool.pool.apply_async(_oracle_config1, ((args.seed, 2000, 100),)) if pool and not args.no_legs else None
    torch.cuda.set_device(dev)
    ctx = P.Context(dev)
    lib = P.lib()
    reqs, probs = make_stream(args, rank)
    dev_inputs = [(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda(), torch.from_numpy(p.a).cuda(),
                   torch.from_numpy(p.b).cuda()) for p in probs]
    l2buf = torch.empty(256 << 18, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize()
        if dist:
            td.barrier()

    stream = torch.cuda.Stream()
    srv = None
    if args.engine == "batched":
        srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=args.slots, stream=stream.cuda_stream)

        def engine(host):
            return run_batched(srv, reqs, probs, dev_inputs, args, host)
    else:
        def engine(host):
            return run_serial(ctx, reqs, probs, dev_inputs, args, host)

    for _ in range(args.warmup):
        engine(False)
        flush_l2(l2buf)
    barrier()
    clock = ClockSampler(dev)
    clock.start()
    lib.ot_profile_reset(ctx.handle)
    lib.ot_profile_enable(ctx.handle, 1)
    if srv is not None:
        srv.reset_stats()
        srv.profile(True)
    step_times, results = [], []
    for _ in range(args.steps):
        flush_l2(l2buf)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = engine(False)
        ev1.record(stream)
        barrier()
        step_times.append(ev0.elapsed_time(ev1) / 1e3)
        results.append(res)
    lib.ot_profile_enable(ctx.handle, 0)
    clocks = clock.stop()
    kst = []
    launch_breakdown = None
    if srv is not None:
        srv.profile(False)
        nl = ctypes.c_int64(srv.stats()["launches"])
        kst = [srv.kernel_stats(kind) for kind in range(2)]
        log = srv.launch_log()
        if len(log):
            # fast launches grouped by the number of instances in the lane: share of the kernel time,
            # and entries/s within the group
            launch_breakdown = []
            for lo, hi in ((1, 1), (2, 4), (5, 16), (17, 64), (65, 1 << 30)):
                m = (log[:, 2] >= lo) & (log[:, 2] <= hi)
                if m.any():
                    launch_breakdown.append({"instances": f"{lo}-{hi}" if hi < (1 << 30) else f">={lo}",
                                             "launches": int(m.sum()),
                                             "time_share": float(log[m, 1].sum() / log[:, 1].sum()),
                                             "entries_per_s": float(log[m, 0].sum() / (log[m, 1].sum() / 1e3))})
    else:
        nl = ctypes.c_int64()
        lib.ot_launch_count(ctx.handle, ctypes.byref(nl))
        for kind in range(2):
            n = ctypes.c_int64()
            e = ctypes.c_double()
            ms = ctypes.c_double()
            lib.ot_profile_read(ctx.handle, kind, ctypes.byref(n), ctypes.byref(e), ctypes.byref(ms))
            kst.append((n.value, e.value, ms.value))
    # end to end: host buffers through the C ABI, copies inside the timed region
    e2e_times, e2e_res = [], []
    for _ in range(args.steps):
        flush_l2(l2buf)
        barrier()
        t = time.perf_counter()
        r2 = engine(True)
        barrier()
        e2e_times.append(time.perf_counter() - t)
        e2e_res.append(r2)

    serial = None
    if args.engine == "batched" and args.serial_steps > 0:
        st_t, st_r = [], None
        for _ in range(args.serial_steps):
            flush_l2(l2buf)
            barrier()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st_r = run_serial(ctx, reqs, probs, dev_inputs, args, host=False)
            ev1.record()
            barrier()
            st_t.append(ev0.elapsed_time(ev1) / 1e3)
        serial = {"value": st_r["entries"] / max(st_t), "unit": UNIT, "ms_per_step": 1e3 * max(st_t),
                  "p50_latency_s": float(np.percentile(st_r["latency"], 50)),
                  "p99_latency_s": float(np.percentile(st_r["latency"], 99)),
                  "converged_frac": st_r["converged"] / len(st_r["latency"]),
                  "note": "same requests solved one at a time with ot_solve (no batching); the results are "
                          "bitwise identical to the batched ones, so the certified gaps are equal"}
    t_step = max(step_times)
    entries = sum(r["entries"] for r in results) / len(results)
    if dist:
        t_step, entries_all, e2e_t, e2e_entries = combine_over_ranks(
            td, "cuda", t_step, entries, statistics.median(e2e_times), e2e_res[-1]["entries"])
    else:
        entries_all = entries
        e2e_t = statistics.median(e2e_times)
        e2e_entries = e2e_res[-1]["entries"]
    if rank != 0:
        if srv is not None:
            srv.close()
        if dist:
            td.barrier()
        return
    lat = results[-1]["latency"]
    ttg = results[-1]["ttg"]
    fast_n, fast_e, fast_ms = kst[0]  # the fast iterations' launches (row and column sweeps)
    # DRAM bytes per implicit entry of the persistent fast launch, from one ncu capture of a serving
    # chunk (dram__bytes_read + write: 2.38 GB over 4.52e11 entries); the traffic is split partials
    # written back from L2, which grow with the entries, so it is scaled to this run's average launch
    traffic = FAST_DRAM_BYTES_PER_ENTRY * fast_e / max(fast_n, 1)
    achieved = fast_e / (fast_ms / 1e3) if fast_ms > 0 else None
    peak = peaks_for_roofline(None, clocks)
    legs = {}
    if not args.no_legs:
        legs["time_to_gap"] = run_time_to_gap(P, ctx, args, stream)
        legs["config1"] = run_config1(P, ctx, args, c1_async.get())
    cpu_v, cpu_dt, cpu_done = pool.sample(args, reqs, args.cpu_sample_s)
    pool.close()
    # The throughput stream stops every request at --max-iters so that a timed step stays short; the
    # time-to-gap and latency fields come from the time-to-gap leg, whose requests run under the
    # config's stop rule (--tol-rel certified gap or --ttg-max-iters) when the legs run.
    stream_fields = {
        "requests": args.requests, "max_iters": args.max_iters,
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "time_to_gap_p50_s": float(np.median(ttg)), "time_to_gap_p99_s": float(np.percentile(ttg, 99)),
        "converged_frac": results[-1]["converged"] / len(lat),
        "time_to_gap_converged_p50_s": (float(np.median(results[-1]["ttg_conv"]))
                                        if results[-1]["ttg_conv"] else None),
        "note": "requests that reach max_iters stop there: these latencies and times are capped-run figures"}
    tg = legs.get("time_to_gap")
    headline = ({"time_to_gap_p50_s": tg["time_to_gap_p50_s"], "time_to_gap_p99_s": tg["time_to_gap_p99_s"],
                 "converged_frac": tg["converged_frac"], "p50_latency_s": tg["latency_p50_s"],
                 "p99_latency_s": tg["latency_p99_s"],
                 "time_to_gap_note": f"{tg['requests']} requests of the stream under the stop rule "
                                     f"({args.tol_rel:g} certified relative gap or {tg['max_iters']} iterations); "
                                     "time to gap over the converged requests, latency over all"}
                if tg else {k: stream_fields[k] for k in ("time_to_gap_p50_s", "time_to_gap_p99_s", "converged_frac",
                                                           "p50_latency_s", "p99_latency_s")})
    out = {
        "metric": METRIC, "value": entries_all / t_step, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 exp / f64 potentials", "data": "synthetic",
        "config": {"workload": "serving stream, mixed 32x32/64x64/128x128 grid histograms",
                   "requests": args.requests, "rate_per_s": args.rate,
                   "max_iters": tg["max_iters"] if tg else args.max_iters,
                   "stream_max_iters": args.max_iters,
                   "time_to_gap_requests": tg["requests"] if tg else args.requests,
                   "cert_every": args.cert_every, "tol_rel": args.tol_rel, "eps0": 1.0, "lambda": args.serve_lam,
                   "engine": args.engine, "seed": args.seed, "l2": "flushed between steps (256 MB write)"},
        **headline,
        "stream": stream_fields,
        "serial_baseline": serial,
        "launch_breakdown": launch_breakdown,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "entries/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_basis": "bytes per launch: 5.3e-3 B/entry from an ncu capture of one serving chunk, "
                                      "scaled by the entries of this run's average launch",
                     "kernel": "fast sweeps (one launch per chunk: row and column sweeps of every instance)",
                     "launches": fast_n,
                     "avg_launch_ms": fast_ms / max(fast_n, 1),
                     "peak_basis": "min(128 FP32 lanes / 4 ops, 32 MUFU ex2) per clk per SM x 148 SMs x sm_max_mhz"},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                         "sample": pool.describe(args.cpu_sample_s, cpu_done) + f"; {cpu_dt:.1f} s wall"},
        "e2e": {"value": e2e_entries / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": e2e_res[-1]["h2d"], "d2h_bytes_per_step": e2e_res[-1]["d2h"]},
        "gpu_launches": int(nl.value),
        "clocks": clocks,
    }
    out.update(legs)
    print(json.dumps(out), flush=True)
    if srv is not None:
        srv.close()
    if dist:
        td.barrier()


def run_load(args):
    """Offered-load sweep of the serving stream, for lambda = 1 and 1.99.  The batched capacity
    (requests/s) is the burst rate: every request of the stream submitted at t = 0, requests /
    makespan.  Poisson streams of the same requests at 0.5, 0.8 and 1.0 times that rate then give
    throughput (entries / makespan, wall clock from the first submission to the last result) and
    the p50/p99 latency from arrival to result."""
    import copy
    import torch
    import paper_2609_33814_b300 as P
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=args.slots, stream=stream.cuda_stream)
    runs = {}
    for lam in (1.0, 1.99):
        a2 = copy.copy(args)
        a2.serve_lam = lam

        def stream_at(rate, burst):
            a2.rate, a2.burst = rate, burst
            reqs, probs = make_stream(a2, 0)
            dev = [tuple(torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)) for p in probs]
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = run_batched(srv, reqs, probs, dev, a2, host=False)
            torch.cuda.synchronize()
            return r, time.perf_counter() - t

        stream_at(args.rate, True)  # warm-up: lanes, graphs, plans
        r, wall = stream_at(args.rate, True)
        cap = args.requests / wall
        rows = [{"load": "burst", "rate_per_s": None, "value": r["entries"] / wall, "makespan_s": wall,
                 "p50_latency_s": float(np.percentile(r["latency"], 50)),
                 "p99_latency_s": float(np.percentile(r["latency"], 99)),
                 "converged_frac": r["converged"] / args.requests}]
        for frac in (0.5, 0.8, 1.0):
            r, wall = stream_at(frac * cap, False)
            rows.append({"load": frac, "rate_per_s": frac * cap, "value": r["entries"] / wall, "makespan_s": wall,
                         "p50_latency_s": float(np.percentile(r["latency"], 50)),
                         "p99_latency_s": float(np.percentile(r["latency"], 99)),
                         "converged_frac": r["converged"] / args.requests})
        runs[f"lambda_{lam:g}"] = {"capacity_req_per_s": cap, "runs": rows}
    srv.close()
    out = {"metric": METRIC, "value": runs["lambda_1"]["runs"][-1]["value"], "unit": UNIT, "n_gpus": 1,
           "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 exp / f64 potentials", "data": "synthetic",
           "config": {"workload": "serving stream at offered loads 0.5/0.8/1.0 x the burst capacity, mixed "
                                  "32x32/64x64/128x128 grid histograms", "requests": args.requests,
                      "max_iters": args.max_iters, "cert_every": args.cert_every, "tol_rel": args.tol_rel,
                      "eps0": 1.0, "seed": args.seed},
           "lambdas": runs}
    print(json.dumps(out), flush=True)


def run_transfer(args):
    """Colour transfer at image size (time-budgeted, gap against wall time): n = m = -(--size) RGB
    points (2^20 = 1024 x 1024 pixels) from seeded 8-component mixtures, uniform weights, kappa =
    1 / max pair cost and omega from the device, eps0 = --eta, lambda = --serve-lam, a certificate
    every --cert-every iterations, until the best relative gap reaches --tol-rel, --max-iters or
    --budget-s of wall time (setup included).  --reverse swaps source and target (the backward
    transfer).  SM clocks are sampled during the run, and the final state's next iteration is
    compared with the oracle on sampled rows and columns."""
    import paper_2609_33814_b300 as P
    import oracle as O
    n = -args.size if args.size < 0 else args.size
    prob = I.rgb_problem(n, args.seed)
    if args.reverse:
        prob = I.Problem(prob.y, prob.x, prob.b, prob.a, prob.kappa, prob.omega, prob.name + "_reverse")
    ctx = P.Context(0)
    clock = ClockSampler(0)
    clock.start()
    t0 = time.perf_counter()
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=0.0, omega=0.0, eps0=args.eta, lam=args.serve_lam,
                  precision="mufu", cert_every=args.cert_every, refine_on=args.refine_on)
    setup_s = time.perf_counter() - t0
    curve, k, rel = [], 0, float("inf")
    while k < args.max_iters and time.perf_counter() - t0 < args.budget_s and rel > args.tol_rel:
        res = S.step(args.cert_every)
        k += args.cert_every
        rel = (res["U_best"] - res["L_best"]) / res["U_best"]
        curve.append({"iter": k, "wall_s": time.perf_counter() - t0, "U_best": res["U_best"],
                      "L_best": res["L_best"], "rel_gap": rel})
    wall = time.perf_counter() - t0
    clocks = clock.stop()
    kappa, omega = S.cost()
    # the next iteration from the final state against the oracle, sampled rows and columns
    lb, lbp = S.get(P.OT_LOG_BETA), S.get(P.OT_LOG_BETA_PREV)
    lbt = lb + (lb - lbp) / args.serve_lam
    eps = O.eps_schedule(args.eta, args.serve_lam, k)
    S.step(1)
    lah, lbh = S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT)
    rng = np.random.default_rng(args.seed)
    rows = np.sort(rng.choice(n, 8, replace=False))
    cols = np.sort(rng.choice(n, 8, replace=False))
    a = prob.a / prob.a.sum()
    b = prob.b / prob.b.sum()
    ref_r = np.log(a[rows]) - O.row_lse_sampled(rows, prob.x, prob.y, lbt, kappa, eps)
    ref_c = np.log(b[cols]) - O.row_lse_sampled(cols, prob.y, prob.x, lah, kappa, eps)
    scale = max(np.abs(eps * lah).max(), np.abs(eps * (lbh - np.log(b))).max())
    err_log = max(np.abs(lah[rows] - ref_r).max(), np.abs(lbh[cols] - ref_c).max())
    parity = {"iter": k + 1, "eps": eps, "rows": 8, "cols": 8, "max_err_log_units": float(err_log),
              "max_err_cost_rel": float(eps * err_log / scale)}
    S.close()
    entries = 2.0 * n * n * k
    out = {"metric": "time to certified relative gap (colour transfer); implicit entries/s", "value": wall,
           "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 exp / f64 potentials, compensated certificates", "data": "synthetic",
           "config": {"workload": f"colour transfer, n = m = {n} RGB points (seeded 8-component mixtures)",
                      "direction": "backward" if args.reverse else "forward",
                      "eps0": args.eta, "lambda": args.serve_lam, "cert_every": args.cert_every,
                      "tol_rel": args.tol_rel, "budget_s": args.budget_s, "kappa": kappa, "omega": omega,
                      "refine_on": args.refine_on},
           "setup_s": setup_s, "iters": k, "final_rel_gap": rel, "entries_per_s": entries / (wall - setup_s),
           "reached_tol": rel <= args.tol_rel, "curve": curve, "final_state_parity": parity, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_project(args):
    """Barycentric projection and marginal errors (ot_plan_project) of one solved instance: implicit
    entries/s over the row pass (with the d projection sums) and the column pass, 2 n m per call."""
    import torch
    import paper_2609_33814_b300 as P
    prob = I.grid_problem(args.size, args.seed) if args.size > 0 else I.rgb_problem(-args.size, args.seed)
    ctx = P.Context(0)
    dev = [torch.from_numpy(v).cuda() for v in (prob.x, prob.y, prob.a, prob.b)]
    S = ctx.state(*dev, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0 if args.size > 0 else 0.1,
                  precision="mufu", cert_every=args.iters)
    S.step(args.iters)  # one certificate iteration: the plan of the best certificate exists
    for _ in range(args.warmup):
        S.project(P.OT_PLAN_BEST)
    clock = ClockSampler(0)
    clock.start()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, _, _, err = S.project(P.OT_PLAN_BEST)
        times.append(time.perf_counter() - t)
    clocks = clock.stop()
    t_call = statistics.median(times)
    entries = 2.0 * prob.n * prob.m
    d = prob.d
    # FP32 lane operations per entry (float-float exponent 8 + 11 d, maximum, sum; d projection FMAs on
    # the row pass), averaged over the two passes
    ops = ((9 + 12 * d) + (9 + 11 * d)) / 2.0
    peak = 128.0 / ops * 148 * (clocks.get("sm_max_mhz") or 2032.0) * 1e6
    out = {"metric": "implicit entries/s, barycentric projection and marginal errors", "value": entries / t_call,
           "unit": "entries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_call, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 float-float exponent, f32 Kahan sums", "data": "synthetic",
           "config": {"workload": f"{'grid %dx%d' % (args.size, args.size) if args.size > 0 else 'rgb %d' % -args.size}"
                                  f" d={d}, plan of the best certificate", "n": prob.n, "m": prob.m,
                      "timing": "wall time of ot_plan_project (its temporary allocation and result copies included)"},
           "roofline": {"bound": "alu", "achieved": entries / t_call, "peak": peak, "unit": "entries/s",
                        "frac": entries / t_call / peak, "traffic": None,
                        "peak_basis": f"128 FP32 lanes / {ops:.1f} ops per entry per clk per SM x 148 SMs x sm_max_mhz"},
           "marginal_errors": err, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_arms(args):
    """Batched O-BDRS arms at equal certified gap: 8 uneven instances (5 x 256^2, 3 x 512^2 grids,
    classes cycling) in one server lane per arm, each run until its best certified relative gap is at
    most --tol-rel.  Arms: MUFU exp2, the FMA-polynomial split and full polynomial, and FP64 (whose
    time to gap is extrapolated from one measured iteration and the MUFU arm's iteration counts:
    a full FP64 run at these sizes takes hours)."""
    import torch
    import paper_2609_33814_b300 as P
    sizes = [256, 512, 256, 512, 256, 256, 512, 256]
    classes = ["uniform", "gaussmix", "cauchy", "sparse"]
    probs = [I.grid_problem(s, args.seed + i, classes[i % 4], classes[(i + 1) % 4]) for i, s in enumerate(sizes)]
    dev = [[torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)] for p in probs]
    ctx = P.Context(0)
    lam = args.lam
    arms = {}
    clock = ClockSampler(0)
    clock.start()
    mufu_iters = None
    for arm in ("mufu", "split", "poly"):
        srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=16)
        srv.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [srv.submit(*d, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15, eps0=1.0, lam=lam,
                          max_iters=args.max_iters, cert_every=args.cert_every, tol_rel=args.tol_rel, precision=arm)
               for d, p in zip(dev, probs)]
        res = [srv.wait(r, 3600.0)[2] for r in ids]
        wall = time.perf_counter() - t0
        n, e, ms = srv.kernel_stats(0)
        srv.close()
        iters = [r["iters"] for r in res]
        if arm == "mufu":
            mufu_iters = iters
        arms[arm] = {"fast_entries_per_s": e / ms * 1e3 if ms else None, "time_to_gap_s": wall,
                     "iters": iters, "gap_rel": [r["gap_rel"] for r in res],
                     "reached": all(r["stop"] == "tol" for r in res)}
    # FP64: one iteration of a 256^2 instance for the rate
    p0 = probs[0]
    S = ctx.state(p0.x, p0.y, p0.a, p0.b, cost_scale=p0.kappa, omega=p0.omega, eps0=1.0, lam=lam, precision="fp64",
                  cert_every=0)
    S.step(1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    S.step(1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    S.close()
    fp64_rate = 2.0 * p0.n * p0.m / dt
    work = sum(2.0 * p.n * p.m * k for p, k in zip(probs, mufu_iters))
    arms["fp64"] = {"fast_entries_per_s": fp64_rate, "time_to_gap_s": work / fp64_rate, "extrapolated": True,
                    "iters": mufu_iters}
    clocks = clock.stop()
    out = {"metric": "time to certified gap, batch of 8 uneven O-BDRS instances (MUFU arm)",
           "value": arms["mufu"]["time_to_gap_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "per arm", "data": "synthetic",
           "config": {"workload": "5 x 256^2 + 3 x 512^2 grid histograms, classes uniform/gaussmix/cauchy/sparse",
                      "lambda": lam, "eps0": 1.0, "tol_rel": args.tol_rel, "cert_every": args.cert_every,
                      "max_iters": args.max_iters},
           "arms": arms, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_ablation(args):
    """The row-update ablation (App. G "Momentum and Kernel Ablation") on an instance with a closed-form
    p*: a cloud of quantised RGB colours and its translate by v (p* = kappa ||v||^2).  For each method
    the dual lower bound L = <r, f> + <c, g> of Prop. 3 is formed from the state after each checkpoint
    (valid for every method: its column update makes B = c / (K^T A)); reported: the relative dual gap
    (p* - L) / p* per checkpoint and the sweep throughput."""
    import torch
    import paper_2609_33814_b300 as P
    n = args.n_points
    x = np.round(I.rgb_cloud(n, args.seed).astype(np.float64) * 1024.0) / 1024.0
    v = np.array([52.0, -31.0, 17.0]) / 1024.0
    y = (x + v).astype(np.float32)
    x = x.astype(np.float32)
    a = np.full(n, 1.0 / n)
    kappa = 1.0 / 3.0
    pstar = kappa * float(v @ v)
    ctx = P.Context(0)
    checkpoints = [50, 200, 800]
    methods = {}
    for alg in ("bdrs", "as", "as_momentum", "as_current", "das"):
        S = ctx.state(x, y, a, a, cost_scale=kappa, omega=1.0, eps0=args.eta, lam=1.0, precision="mufu",
                      cert_every=0, algorithm=alg)
        gaps, k, tsum = {}, 0, 0.0
        for c in checkpoints:
            torch.cuda.synchronize()
            t = time.perf_counter()
            S.step(c - k)
            torch.cuda.synchronize()
            tsum += time.perf_counter() - t
            k = c
            eps = args.eta / (k - 1 + 1.0)
            L = float(a @ (eps * S.get(P.OT_LOG_ALPHA_HAT)) + a @ (eps * (S.get(P.OT_LOG_BETA_HAT) - np.log(a))))
            gaps[c] = (pstar - L) / pstar
        S.close()
        methods[alg] = {"rel_dual_gap": gaps, "entries_per_s": 2.0 * n * n * checkpoints[-1] / tsum}
    out = {"metric": "relative dual gap (p* - L)/p* per row-update method", "value": methods["bdrs"]["rel_dual_gap"][800],
           "unit": "relative", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 exp / f64 potentials", "data": "synthetic",
           "config": {"workload": f"quantised RGB cloud of {n} points and its translate (p* = kappa |v|^2)",
                      "eta": args.eta, "lambda": 1.0, "checkpoints": checkpoints}, "methods": methods}
    print(json.dumps(out), flush=True)


def transport_lp(a, b, C) -> float:
    """Exact p* of a small non-uniform instance: the transport LP, solved by scipy's HiGHS.  The
    n + m equalities have rank n + m - 1, so the last is dropped (a total-mass mismatch of a few
    ulps would otherwise make the presolve declare the system infeasible)."""
    from scipy.optimize import linprog
    from scipy.sparse import identity, kron, vstack
    n, m = C.shape
    A_eq = vstack([kron(identity(n), np.ones((1, m))), kron(np.ones((1, n)), identity(m))]).tocsr()[:-1]
    res = linprog(C.ravel(), A_eq=A_eq, b_eq=np.concatenate([a, b])[:-1], bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"transport LP: {res.message}")
    return float(res.fun)


def delay_instances(args):
    """(x, y, a, b, kappa, p*) per instance pair of the delay workload, with the exact p*."""
    from scipy.optimize import linear_sum_assignment
    out = []
    for i in range(args.instances):
        if args.delay_set == "clouds":
            n = 1024
            x = I.rgb_cloud(n, args.seed + 2 * i)[:, :2].copy()
            y = I.rgb_cloud(n, args.seed + 2 * i + 1)[:, :2].copy()
            C = ((x[:, None, :].astype(np.float64) - y[None, :, :]) ** 2).sum(-1)
            kappa = 1.0 / C.max()
            rows, cols = linear_sum_assignment(C)
            w = np.full(n, 1.0 / n)
            out.append((x, y, w, w, kappa, kappa * C[rows, cols].sum() / n))
        else:
            classes = I.HIST_CLASSES
            p = I.grid_problem(16, args.seed + 2 * i, classes[i % len(classes)], classes[(i + 1) % len(classes)])
            a = np.maximum(p.a, 1e-15)
            a = a / a.sum()
            b = np.maximum(p.b, 1e-15)
            b = b / b.sum()
            C = p.kappa * ((p.x[:, None, :].astype(np.float64) - p.y[None, :, :]) ** 2).sum(-1)
            out.append((p.x, p.y, p.a, p.b, p.kappa, transport_lp(a, b, C)))
    return out


def run_delay(args):
    """Certification delay (the paper's D(tau) = k_cert(tau) / k_oracle(tau)).  Instances: pairs of
    uniform-weight clouds, whose exact p* is an assignment problem (scipy's linear_sum_assignment), or
    16x16 grid histograms of the four classes (zero masses floored at 1e-15), whose exact p* is the
    transport LP (scipy's HiGHS).  Each runs with a certificate every 10 iterations up to 10^4
    iterations; k_oracle(tau) = first certificate iteration with U_best - p* <= tau, k_cert(tau) =
    first with U_best - L_best <= tau (additive tau on costs normalised to [0, 1])."""
    import paper_2609_33814_b300 as P
    count, budget, every = args.instances, 10000, 10
    taus = [1e-2, 1e-3, 1e-4]
    ctx = P.Context(0)
    insts = delay_instances(args)
    out_methods = {}
    for name, lam in (("bdrs", 1.0), ("obdrs_1.99", 1.99)):
        delays = {t: [] for t in taus}
        certified = {t: 0 for t in taus}
        for x, y, a, b, kappa, pstar in insts:
            S = ctx.state(x, y, a, b, cost_scale=kappa, omega=1.0, zero_mass_floor=1e-15, eps0=1.0, lam=lam,
                          precision="mufu", cert_every=every)
            k_or = {t: None for t in taus}
            k_ce = {t: None for t in taus}
            k = 0
            while k < budget and any(v is None for v in k_ce.values()):
                res = S.step(every)
                k += every
                for t in taus:
                    if k_or[t] is None and res["U_best"] - pstar <= t:
                        k_or[t] = k
                    if k_ce[t] is None and res["U_best"] - res["L_best"] <= t:
                        k_ce[t] = k
            S.close()
            for t in taus:
                if k_ce[t] is not None and k_or[t] is not None:
                    delays[t].append(k_ce[t] / k_or[t])
                    certified[t] += 1
        out_methods[name] = {f"{t:g}": {"median_delay": float(np.median(delays[t])) if delays[t] else None,
                                        "max_delay": float(np.max(delays[t])) if delays[t] else None,
                                        "certified": certified[t], "of": count} for t in taus}
    if args.delay_set == "clouds":
        workload = f"{count} pairs of 1024-point 2-D clouds (colour-mixture marginals), uniform weights"
        exact = "exact assignment (scipy linear_sum_assignment)"
    else:
        workload = f"{count} pairs of 16x16 grid histograms, classes cycled over the four histogram classes"
        exact = "exact transport LP (scipy HiGHS)"
    out = {"metric": "certification delay D(tau) = k_cert / k_oracle (median over instances)",
           "value": out_methods["bdrs"]["0.01"]["median_delay"], "unit": "ratio", "n_gpus": 1, "steps": 1,
           "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 exp / f64 potentials, compensated certificates", "data": "synthetic",
           "config": {"workload": workload, "eps0": 1.0, "cert_every": every, "budget": budget, "pstar": exact},
           "methods": out_methods}
    print(json.dumps(out), flush=True)


def run_precision(args):
    """The FP32 exponent of the fast iterations against a compensated one, per result (App. G,
    "Floating-point evaluation"), on the serving stream's requests under the config's stop rule.

    Every request of the stream is submitted at t = 0 in OT_EXP_MUFU with the stop rule (--tol-rel
    certified gap, --max-iters cap) and broken down by grid size and histogram class.  A sample of
    --study-n requests (those that did not certify first, largest grids first) is then run again
    in each arm of --study-arms, to the same cap: ``comp`` is OT_FP32_COMP (float-float exponent on
    every iteration, the FP64-equivalent reference), ``centred`` is OT_EXP_MUFU on the same grid
    translated by (s - 1) / 2 (exact for integer pixel coordinates; the cost is unchanged), and
    ``mufu`` repeats the default."""
    import torch
    import paper_2609_33814_b300 as P
    ctx = P.Context(0)
    stream = torch.cuda.Stream()
    args.burst = True
    reqs, probs = make_stream(args, 0)

    def run_set(idx, precision, centre, refine=(0.0, 0.0)):
        srv = P.Server(ctx, hbm_budget_bytes=64 << 30, max_slots=max(len(idx), 1), stream=stream.cuda_stream)
        prm = dict(solve_params(args), precision=precision, refine_on=refine[0], refine_tol=refine[1])
        t0 = time.perf_counter()
        ids = []
        for i in idx:
            p = probs[i]
            x, y = p.x, p.y
            if centre:
                o = np.float32(0.5 * (reqs[i].s - 1))
                x, y = x - o, y - o
            ids.append(srv.submit(x, y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15, **prm))
        out = {}
        for i, rid in zip(idx, ids):
            f, g, res = srv.wait(rid, -1.0)
            out[i] = {"iters": int(res["iters"]), "stop": res["stop"], "gap_rel": res["gap_rel"],
                      "U_best": res["U_best"], "L_best": res["L_best"],
                      "latency_s": res["latency_s"] - res["queue_s"]}
        wall = time.perf_counter() - t0
        srv.close()
        return out, wall

    base_refine = tuple(float(v) for v in args.study_base.split(":"))
    base, wall0 = run_set(list(range(len(reqs))), "mufu", False, base_refine)
    groups = {}
    for i, r in enumerate(reqs):
        for key in (f"s{r.s}", f"s{r.s}:{r.cls_a}/{r.cls_b}"):
            g = groups.setdefault(key, {"count": 0, "converged": 0, "iters": [], "gap": []})
            g["count"] += 1
            g["converged"] += base[i]["stop"] == "tol"
            g["iters"].append(base[i]["iters"])
            g["gap"].append(base[i]["gap_rel"])
    table = {k: {"count": v["count"], "converged": v["converged"], "median_iters": float(np.median(v["iters"])),
                 "median_best_gap": float(np.median(v["gap"])), "max_best_gap": float(np.max(v["gap"]))}
             for k, v in sorted(groups.items())}
    order = sorted(range(len(reqs)), key=lambda i: (base[i]["stop"] == "tol", -reqs[i].s, i))
    sample = order[:args.study_n]
    arms = {}
    for arm in [a for a in args.study_arms.split(",") if a]:
        # arm names: comp, mufu, centred; a suffix @ON:TOL runs the arm with the fast sweeps'
        # refinement thresholds refine_on = ON, refine_tol = TOL (no suffix: no refinement)
        name, _, ref = arm.partition("@")
        centre = name == "centred"
        refine = tuple(float(v) for v in ref.split(":")) if ref else (0.0, 0.0)
        res, wall = run_set(sample, "comp" if name == "comp" else "mufu", centre, refine)
        arms[arm] = {"wall_s": wall, "results": res}
    rows = []
    for i in sample:
        row = {"s": reqs[i].s, "classes": f"{reqs[i].cls_a}/{reqs[i].cls_b}", "seed": reqs[i].seed,
               "mufu": base[i]}
        for arm, v in arms.items():
            row[arm] = v["results"][i]
        rows.append(row)
    out = {"metric": "certified relative gap and iterations to it, FP32 exponent against compensated",
           "unit": "iterations", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "serving stream requests, burst, mixed 32x32/64x64/128x128 grid histograms",
                      "requests": args.requests, "max_iters": args.max_iters, "cert_every": args.cert_every,
                      "tol_rel": args.tol_rel, "eps0": 1.0, "lambda": args.serve_lam, "seed": args.seed},
           "stream_wall_s": wall0, "converged_frac": sum(b["stop"] == "tol" for b in base.values()) / len(reqs),
           "by_size_class": table, "sample": rows}
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """One resident instance, fast iterations only: entries/s of the sweep kernels alone, after --skip
    untimed iterations (deep in the schedule the fast sweeps refine their dominant terms, see
    ot_params; --refine-on sets its threshold, 0 leaves it off)."""
    import ctypes
    import torch
    import paper_2609_33814_b300 as P
    prob = I.grid_problem(args.size, args.seed) if args.size > 0 else I.rgb_problem(-args.size, args.seed)
    ctx = P.Context(0)
    lib = P.lib()
    dev = [torch.from_numpy(v).cuda() for v in (prob.x, prob.y, prob.a, prob.b)]
    S = ctx.state(*dev, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0 if args.size > 0 else 0.1,
                  precision=args.precision, cert_every=0, refine_on=args.refine_on)
    if args.skip > 0:
        S.step(args.skip)
    refined0 = S.counters()["tiles_refined"]
    for _ in range(args.warmup):
        S.step(args.iters)
    clock = ClockSampler(0)
    clock.start()
    lib.ot_profile_reset(ctx.handle)
    lib.ot_profile_enable(ctx.handle, 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        S.step(args.iters)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    lib.ot_profile_enable(ctx.handle, 0)
    clocks = clock.stop()
    n = ctypes.c_int64(); e = ctypes.c_double(); ms = ctypes.c_double()
    tot_n, tot_e, tot_ms = 0, 0.0, 0.0
    lib.ot_profile_read(ctx.handle, 0, ctypes.byref(n), ctypes.byref(e), ctypes.byref(ms))  # fast iterations
    tot_n, tot_e, tot_ms = n.value, e.value, ms.value
    achieved = tot_e / (tot_ms / 1e3)
    d = prob.d
    peak = min(128.0 / (d + 2), 32.0) * 148 * (clocks.get("sm_max_mhz") or 2032.0) * 1e6
    out = {"metric": "implicit entries/s per dual sweep (one resident instance)", "value": achieved,
           "unit": "entries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
           "config": {"workload": f"{'grid %dx%d' % (args.size, args.size) if args.size > 0 else 'rgb %d' % -args.size}"
                                  f" d={d}, {args.iters} iterations per step", "n": prob.n, "m": prob.m,
                      "skip": args.skip, "refine_on": args.refine_on},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "entries/s",
                        "frac": achieved / peak, "traffic": None, "launches": tot_n,
                        "avg_launch_ms": tot_ms / max(tot_n, 1)},
           "tiles_refined": S.counters()["tiles_refined"] - refined0,
           "clocks": clocks}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.workload == "sweep":
        run_sweep(args)
        return
    if args.workload == "project":
        run_project(args)
        return
    if args.workload == "arms":
        run_arms(args)
        return
    if args.workload == "ablation":
        run_ablation(args)
        return
    if args.workload == "load":
        run_load(args)
        return
    if args.workload == "transfer":
        run_transfer(args)
        return
    if args.workload == "delay":
        run_delay(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world)


if __name__ == "__main__":
    main()
