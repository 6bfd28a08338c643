#!/usr/bin/env python3
"""Benchmark of the convex-clustering path solver on one GB300 (or N replicas).

One step = the whole hot path on one synthetic problem: the kNN Gaussian-kernel
weights on the GPU, then the warm-started gamma path (all MM iterations,
per-gamma outputs and labels).  Default workload, "genotype-like":
n = 1000 individuals x p = 10000 SNPs from 5 Balding-Nichols populations
(Fst = 0.05, ancestral frequency U(0.05, 0.5)), codes standardised on the
observed entries, 5 % of entries missing; kNN k = 10 with phi = 1/median d^2
and weights normalised to sum 1; 50 gamma log-spaced over [0.03, 3] x the
two-point fusion scale (from before the first fusion to past complete fusion
within the graph's components).  The data are synthetic stand-ins for the paper's
genotype sets.

Metric: edge-updates/s = sum over gammas of |E| * p * (MM iterations), per
second of device time, inputs resident in HBM (value); the same through the
C ABI with host inputs and host outputs, copies inside the timed region (e2e).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ccx|reference]
For N > 1 launch with torchrun: each rank solves its own replica (weak scaling).
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

import synth  # noqa: E402

METRIC = "edge-updates/s (edges*p*iters)"
UNIT = "edge-updates/s"


def workload(name: str):
    if name == "genotype":
        X, mask, _ = synth.genotype_like(1000, 10000, 5, seed=1, fst=0.05, frac_missing=0.05)
        # Anderson mixing: the path has 17 gammas before the first fusion, where it cuts iterations
        # (history 8 measured fastest among 3, 5, 6, 7, 8, 12 and 16)
        return dict(X=X, mask=mask, k=10, phi_auto=True, normalize=True, n_gamma=50, lo=3e-2, hi=3.0, anderson=8,
                    desc="genotype-like n=1000 p=10000, 5 pops Balding-Nichols Fst=0.05, 5% missing, "
                         "kNN k=10 phi=1/median d2 normalised, 50 gamma in [0.03,3]*gamma0")
    if name == "expression":
        X, _ = synth.expression_like(100, 20000, 3, 500, seed=2)
        return dict(X=X, mask=None, k=99, phi_auto=True, normalize=True, n_gamma=40, lo=3e-2, hi=3.0,
                    desc="expression-like n=100 p=20000, all 4950 pairs, phi=1/median d2 normalised, "
                         "40 gamma in [0.03,3]*gamma0")
    if name == "plain":
        X, _ = synth.gaussian_mixture(200, 10, 4, seed=0)
        return dict(X=X, mask=None, k=10, phi=0.5, phi_auto=False, normalize=False, n_gamma=20, fixed=(1e-3, 1e1),
                    precision=1, desc="plain n=200 p=10 4 Gaussian clusters, kNN k=10 w=exp(-0.5 d2), "
                                      "20 gamma 1e-3..1e1, FP64 path")
    raise SystemExit(f"unknown workload {name}")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 4 + k and "Active" in r[4 + k]
                          and "Not" not in r[4 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist.get_rank(), ws, dist


def dist_max(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- oracle timing
def oracle_sample(W, seconds: float, gammas, edges):
    """Literal FP64 MM steps of the oracle on this workload for about `seconds`."""
    import oracle as O
    X = W["X"].astype(np.float64)
    ei, ej, w = edges
    G = O.EdgeGraph(X.shape[0], ei, ej, w)
    Y0 = O.fill_missing(X, W["mask"])
    mu = float(gammas[len(gammas) // 2])
    rho, eps = O.pd_constants(Y0, G.w, mu)
    U, V = Y0.copy(), np.zeros((G.m, X.shape[1]))
    t0 = time.perf_counter()
    steps = 0
    while True:
        U, V, _, _ = O.mm_step(U, V, X, W["mask"], G, mu, rho, eps)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 1000:
            break
    return G.m * X.shape[1] * steps / el, steps, el


def oracle_edges(W):
    import oracle as O
    ei, ej, w, _, _ = O.knn_gaussian_weights(W["X"].astype(np.float64), W["mask"], W["k"],
                                             "auto" if W.get("phi_auto") else W.get("phi", 0.0), W["normalize"])
    return ei, ej, w


def run_config(W, m: int, ws: int):
    """The `config` object of the JSON line; both arms print the same one."""
    n, p = W["X"].shape
    ld = (p + 31) // 32 * 32
    # device bytes the iteration touches: X, Y_0, two (hi, lo) slots of A, two Delta slots,
    # the output staging row block, and the two missing-data offsets when there is a mask
    ws_mb = n * ld * (4 * (1 + 1 + 4 + 2 + 1) + (8 if W["mask"] is not None else 0)) / 1e6
    return {"workload": W["desc"], "n": n, "p": p, "edges": int(m), "gammas": W["n_gamma"],
            "l2": f"working set of the iteration ~{ws_mb:.0f} MB; a 256 MB buffer is written between timed "
                  "steps to flush L2", "parallelism": f"replicas x{ws}"}


def source_sha(path: str) -> str:
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def stored_traffic(workload: str):
    """(bytes per launch, note) of the iteration kernel from the committed ncu summary, or
    (None, why) when it is missing or was taken on a different kernel source."""
    tfile = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(tfile):
        return None, "no ncu capture for this workload"
    try:
        t = json.load(open(tfile))
    except Exception:
        return None, "unreadable capture record"
    src = os.path.join(ROOT, "paper_1409_2065_gb300", "csrc", "pd_kernels.cu")
    if t.get("source_sha256") != source_sha(src):
        return None, "the kernel source changed since the ncu capture"
    return t.get("bytes_per_launch"), f"from profile: {t.get('source', 'ncu capture')}"


def gamma_grid(W, g0):
    if "fixed" in W:
        return synth.log_grid(W["fixed"][0], W["fixed"][1], W["n_gamma"])
    return synth.log_grid(W["lo"] * g0, W["hi"] * g0, W["n_gamma"])


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    W = workload(args.workload)
    import oracle as O
    t = time.perf_counter()
    edges = oracle_edges(W)
    g0 = O.fusion_scale(W["X"], W["mask"], *edges)
    gammas = gamma_grid(W, g0)
    vals = []
    for s in range(args.warmup + args.steps):
        v, steps, el = oracle_sample(W, args.ref_seconds, gammas, edges)
        if s >= args.warmup:
            vals.append(v)
    val = statistics.median(vals)
    cores = os.cpu_count()
    sample = f"{args.ref_seconds:.0f} s of literal FP64 MM steps (exact projection) per step at the middle gamma"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": args.ref_seconds * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(W, int(edges[0].size), ws),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": time.perf_counter() - t}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batched problems
def batch_specs(count, nmax, pmax, seed=3):
    """Sizes of the batched workload: n ~ U[50, nmax], p ~ U[10, pmax], 2-8 Gaussian clusters
    (means ~ N(0, 9 I), noise N(0, I)), problem i drawn with seed 1000 * seed + i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(1000 * seed + i)
        n = int(rng.integers(50, nmax + 1))
        p = int(rng.integers(10, pmax + 1))
        k = int(rng.integers(2, 9))
        X, _ = synth.gaussian_mixture(n, p, k, seed=1000 * seed + i)
        out.append(X)
    return out


def run_batch(args, ccx, torch, rank):
    """Batched workload: the same problems solved (1) one call after another (the plain
    per-launch path), (2) together with ccx_solve_batch on the default grid (results
    must be bit-identical to (1)), (3) together after ccx_tune_grid picked each
    problem's grid (results agree with (1) within the FP32 parity bar)."""
    Xs = batch_specs(args.batch, args.batch_nmax, args.batch_pmax)

    def make():
        probs = []
        for X in Xs:
            pr = ccx.Problem(torch.from_numpy(X).cuda())
            pr.build_knn(10, phi_auto=True, normalize=True)
            probs.append(pr)
        return probs

    probs = make()
    grids = [synth.log_grid(0.03 * pr.fusion_scale(), 3.0 * pr.fusion_scale(), args.batch_gammas) for pr in probs]
    opts = ccx.opts_default()
    opts.anderson = args.anderson or 0          # the same options in every arm
    # (1) one call per problem, one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [pr.solve_path(g, opts, device=True) for pr, g in zip(probs, grids)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    iters = sum(s["iters"] for r in seq for s in r[2])
    conv_seq = all(s["converged"] in (1, 2) for r in seq for s in r[2])
    # (2) together, default grid
    for pr in probs:
        pr.reset_path()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Us, Ls, stats, status, _ = ccx.solve_batch(probs, grids, opts, device=True, max_active=args.batch_active)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    same = all(torch.equal(Us[i], seq[i][0]) and torch.equal(Ls[i], seq[i][1]) for i in range(len(probs)))
    del Us, Ls
    # (3) together, grids from the autotuner
    for pr in probs:
        pr.reset_path()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_min = max(1, 152 // max(1, args.batch_active))
    tuned = [pr.tune_grid(g_min)[0] for pr in probs]
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    Ut, Lt, stt, status_t, _ = ccx.solve_batch(probs, grids, opts, device=True, max_active=args.batch_active)
    torch.cuda.synchronize()
    t_tb = time.perf_counter() - t0
    rel = max(float(torch.linalg.vector_norm(Ut[i][g] - seq[i][0][g]) / torch.linalg.vector_norm(seq[i][0][g]))
              for i in range(len(probs)) for g in range(len(grids[i])))
    lab_same = sum(int(torch.equal(Lt[i], seq[i][1])) for i in range(len(probs)))
    conv_t = all(s["converged"] in (1, 2) for st_ in stt for s in st_)
    sz = [X.shape for X in Xs]
    line = {"metric": "gamma-path solves/s", "workload": f"{args.batch} problems, n~U[50,{args.batch_nmax}], "
            f"p~U[10,{args.batch_pmax}], 2-8 clusters, kNN k=10, {args.batch_gammas} gammas in [0.03,3]*gamma0",
            "plain_one_call_per_problem": len(probs) / t_seq, "batched": len(probs) / t_bat,
            "batched_tuned_grids": len(probs) / (t_tb + t_tune),
            "speedup": t_seq / t_bat, "speedup_tuned_incl_tuning": t_seq / (t_tb + t_tune),
            "seconds_plain": t_seq, "seconds_batched": t_bat, "seconds_tuned": t_tb, "seconds_tuning": t_tune,
            "tuned_grids": tuned, "max_active": args.batch_active, "mm_iterations_plain": int(iters),
            "anderson": int(opts.anderson),
            "sum_np": int(sum(n * p for n, p in sz)), "identical_results": bool(same),
            "tuned_max_rel_diff_U": rel, "tuned_problems_with_identical_labels": lab_same,
            "all_converged": bool(conv_seq and conv_t and all(s == 0 for s in status + status_t)),
            "dtype": "f32", "data": "synthetic"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args, ccx, torch, rank):
    """Serving workload: Poisson arrivals of jobs from the batched size distribution at each
    rate of --serve, served by ccx_server with continuous batching and, on the same jobs and
    arrival times, one job at a time (max_active = 1); p50/p99 latency and solves/s."""
    rates = [float(r) for r in str(args.serve).split(",")]
    Xs = batch_specs(args.serve_jobs, args.batch_nmax, args.batch_pmax, seed=4)

    def arm(max_active, gaps):
        probs = []
        for X in Xs:
            pr = ccx.Problem(torch.from_numpy(X).cuda())
            pr.build_knn(10, phi_auto=True, normalize=True)
            probs.append(pr)
        grids = [synth.log_grid(0.03 * pr.fusion_scale(), 3.0 * pr.fusion_scale(), args.batch_gammas)
                 for pr in probs]
        torch.cuda.synchronize()
        srv = ccx.Server(max_active=max_active)
        arrive, done, results = [0.0] * len(Xs), [0.0] * len(Xs), [None] * len(Xs)
        codes = [None] * len(Xs)

        def waiter(i, t):
            st, U, L, stats = srv.wait(t, -1)
            done[i] = time.perf_counter()
            results[i] = (U, L)
            codes[i] = st

        threads = []
        t0 = time.perf_counter()
        due = t0
        for i, pr in enumerate(probs):
            due += gaps[i]
            time.sleep(max(0.0, due - time.perf_counter()))
            arrive[i] = time.perf_counter()
            th = threading.Thread(target=waiter, args=(i, srv.submit(pr, grids[i], device=True)))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        wall = max(done) - t0
        srv.close()
        lat = sorted(d - a for d, a in zip(done, arrive))
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
        for pr in probs:
            pr.close()
        return {"p50_s": q(0.5), "p99_s": q(0.99), "solves_per_s": len(Xs) / wall, "wall_s": wall,
                "all_ok": all(c == 0 for c in codes)}, results

    per_rate = []
    for r_i, rate in enumerate(rates):
        gaps = np.random.default_rng(4 + r_i).exponential(1.0 / rate, size=len(Xs))
        served, r1 = arm(args.serve_active, gaps)
        plain, r2 = arm(1, gaps)
        same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(r1, r2))
        per_rate.append({"rate_jobs_per_s": rate, "continuous_batching": served, "one_at_a_time": plain,
                         "speedup_solves_per_s": served["solves_per_s"] / plain["solves_per_s"],
                         "identical_results": bool(same)})
    line = {"metric": "served gamma-path solves/s and latency",
            "workload": f"{len(Xs)} jobs per rate, Poisson arrivals, n~U[50,{args.batch_nmax}], "
                        f"p~U[10,{args.batch_pmax}], 2-8 clusters, kNN k=10, {args.batch_gammas} gammas in "
                        "[0.03,3]*gamma0", "max_active": args.serve_active, "rates": per_rate,
            "dtype": "f32", "data": "synthetic"}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ccx", choices=["ccx", "reference"])
    ap.add_argument("--workload", default="genotype", choices=["genotype", "expression", "plain"])
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=0, metavar="P",
                    help="instead of the default step: P independent problems from the batched-workload size "
                         "distribution (scaled by --batch-nmax/--batch-pmax), solved one call after another and "
                         "then together with ccx_solve_batch; prints the two solve rates")
    ap.add_argument("--serve", type=str, default="", metavar="RATES",
                    help="instead of the default step: for each comma-separated rate, Poisson arrivals of "
                         "--serve-jobs jobs at that many jobs/s (sizes as --batch), served by ccx_server with "
                         "continuous batching and, for comparison, one job at a time; prints p50/p99 latency "
                         "and solve rates")
    ap.add_argument("--serve-jobs", type=int, default=64)
    ap.add_argument("--serve-active", type=int, default=32, help="jobs the server runs at once")
    ap.add_argument("--batch-nmax", type=int, default=2000)
    ap.add_argument("--batch-pmax", type=int, default=5000)
    ap.add_argument("--batch-gammas", type=int, default=30)
    ap.add_argument("--batch-active", type=int, default=32, help="problems with work queued at once")
    ap.add_argument("--min-k", type=int, default=0, metavar="KMAX",
                    help="instead of the default step: time the search for the smallest k <= KMAX whose kNN "
                         "graph of the workload is connected, on the GPU and with the oracle")
    ap.add_argument("--composite", type=float, default=-1.0, metavar="ALPHA",
                    help="instead of the default step: time the kNN weights on the composite distance "
                         "ALPHA * genetic + (1 - ALPHA) * great-circle distance (sampling sites synthetic: one "
                         "site per population plus 2-degree jitter), on the GPU and with the oracle")
    ap.add_argument("--pc", type=int, default=0, metavar="Q",
                    help="instead of the default step: time the Q principal axes of the workload on the GPU and "
                         "with the oracle, and the projected path against the full path through host buffers")
    ap.add_argument("--gram-compare", action="store_true",
                    help="instead of the default step: time the kNN weights of the workload with the Gram on "
                         "TF32 and BF16 tensor cores and on FP32 CUDA cores, and check the edge sets agree")
    ap.add_argument("--slice-variant", type=int, default=0, choices=[0, 1, 2],
                    help="staging of the iteration kernel's slices: 0 automatic, 1 double buffer where it fits, "
                         "2 single buffer")
    ap.add_argument("--anderson", type=int, default=None, metavar="M",
                    help="Anderson mixing of the MM map over M map outputs while the previous gamma had no "
                         "fused edge (0: off, the plain restart rule throughout); default: the workload's "
                         "setting (8 for genotype, whose path has many gammas before fusion; 0 for the others)")
    ap.add_argument("--fuse-delta", type=float, default=None, metavar="D",
                    help="relative band around the fusion threshold in which an edge's norm is recomputed "
                         "in double before its fuse decision (library default 1e-5; 0 turns it off)")
    ap.add_argument("--mixing-only", type=int, default=0, metavar="K",
                    help="build the workload, run K individually launched MM iterations with Anderson mixing "
                         "(history --anderson) at the first gamma and print the mean times of the iteration, "
                         "reduction and mixing kernels (K < 320 keeps every iteration mixed)")
    ap.add_argument("--iterations-only", type=int, default=0, metavar="K",
                    help="build the workload, run K individually launched MM iterations at the middle gamma "
                         "and print the two kernels' mean times (a short target for a profiler)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, ws, dist = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
        return

    import torch
    import paper_1409_2065_gb300 as ccx
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.batch:
        run_batch(args, ccx, torch, rank)
        return
    if args.serve:
        run_serve(args, ccx, torch, rank)
        return
    W = workload(args.workload)
    if args.anderson is None:
        args.anderson = W.get("anderson", 0)
    opts = ccx.opts_default()
    opts.slice_variant = args.slice_variant
    opts.anderson = args.anderson
    if args.fuse_delta is not None:
        opts.fuse_delta = args.fuse_delta
    n, p = W["X"].shape
    Xd = torch.from_numpy(W["X"]).cuda()
    Md = torch.from_numpy(W["mask"]).cuda() if W["mask"] is not None else None
    prec = W.get("precision", ccx.CCX_FP32)
    pr = ccx.Problem(Xd, Md, prec)
    pr.build_knn(W["k"], phi=W.get("phi", 0.0), phi_auto=W.get("phi_auto", False), normalize=W["normalize"])
    ei, ej, w = pr.get_edges()
    m = int(ei.size)
    gammas = gamma_grid(W, pr.fusion_scale())
    G = len(gammas)
    if args.composite >= 0.0:
        rng = np.random.default_rng(5)
        pops = 5
        sites = np.c_[rng.uniform(-50, 60, pops), rng.uniform(-180, 180, pops)]
        who = np.arange(n) * pops // n                      # cases are stored population by population
        coords = sites[who] + rng.normal(0.0, 2.0, (n, 2))
        coords[:, 0] = np.clip(coords[:, 0], -90.0, 90.0)
        kw = dict(phi_auto=True, normalize=True, geodesic=True)
        pr.build_knn_composite(W["k"], coords, args.composite, **kw)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr.build_knn_composite(W["k"], coords, args.composite, **kw)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - t0
        ei, ej, w = pr.get_edges()
        import oracle as O
        t0 = time.perf_counter()
        oei, oej, ow, _, _ = O.knn_composite_weights(W["X"].astype(np.float64), W["mask"], coords, args.composite,
                                                     W["k"], "auto", True, True)
        t_ref = time.perf_counter() - t0
        same = bool(np.array_equal(ei, oei) and np.array_equal(ej, oej) and np.allclose(w, ow, rtol=1e-10))
        print(json.dumps({"metric": "seconds per composite-distance kNN weight build", "workload": W["desc"],
                          "alpha": args.composite, "edges": int(ei.size), "gpu_seconds": t_gpu,
                          "oracle_seconds": t_ref, "oracle_cores": os.cpu_count(), "identical_to_oracle": same}),
              flush=True)
        return
    if args.pc:
        pr.principal_axes(args.pc)                          # warm-up (and cached on the problem)
        q2 = 1 if args.pc > 1 else 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        axes, var = pr.principal_axes(q2)                   # a different q forces a recomputation
        axes, var = pr.principal_axes(args.pc)
        torch.cuda.synchronize()
        t_gpu = (time.perf_counter() - t0) / 2.0
        import oracle as O
        t0 = time.perf_counter()
        oaxes, ovar = O.principal_axes(W["X"].astype(np.float64), W["mask"], args.pc)
        t_ref = time.perf_counter() - t0
        sub = gammas[::10]
        pr.reset_path()
        t0 = time.perf_counter()
        pr.solve_path(sub)
        t_full = time.perf_counter() - t0
        pr.reset_path()
        t0 = time.perf_counter()
        pr.solve_path_projected(sub, args.pc)
        t_proj = time.perf_counter() - t0
        print(json.dumps({"metric": "principal axes and projected path", "workload": W["desc"], "q": args.pc,
                          "axes_gpu_seconds": t_gpu, "axes_oracle_seconds": t_ref,
                          "max_abs_axis_diff": float(np.abs(axes - oaxes).max()),
                          "max_rel_var_diff": float(np.max(np.abs(var - ovar) / ovar)),
                          "path_gammas": len(sub), "path_host_outputs_seconds": t_full,
                          "path_projected_seconds": t_proj,
                          "bytes_out_per_gamma_full": int(n * p * 4), "bytes_out_per_gamma_projected": int(n * args.pc * 4)}),
              flush=True)
        return
    if args.gram_compare:
        out = {}
        edges0 = None
        for gram, name in ((0, "tf32_tensor_cores"), (1, "bf16_tensor_cores"), (2, "fp32_cuda_cores")):
            kw = dict(phi=W.get("phi", 0.0), phi_auto=W.get("phi_auto", False), normalize=W["normalize"], gram=gram)
            pr.build_knn(W["k"], **kw)                       # warm-up
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                pr.build_knn(W["k"], **kw)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            e = pr.get_edges()
            if edges0 is None:
                edges0 = e
            same = all(np.array_equal(a, b) for a, b in zip(e, edges0))
            out[name] = {"seconds_median": statistics.median(ts), "edges_identical_to_tf32": bool(same)}
        print(json.dumps({"metric": "seconds per kNN weight build by Gram precision", "workload": W["desc"],
                          "edges": int(edges0[0].size), **out}), flush=True)
        return
    if args.min_k:
        pr.min_connected_k(args.min_k)                      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k_gpu = pr.min_connected_k(args.min_k)
        torch.cuda.synchronize()
        t_gpu = time.perf_counter() - t0
        import oracle as O
        t0 = time.perf_counter()
        k_ref = O.min_connected_k(W["X"].astype(np.float64), W["mask"], args.min_k)
        t_ref = time.perf_counter() - t0
        print(json.dumps({"metric": "seconds to the smallest connected k", "workload": W["desc"], "k_max": args.min_k,
                          "k": k_gpu, "oracle_k": k_ref, "gpu_seconds": t_gpu, "oracle_seconds": t_ref,
                          "oracle_cores": os.cpu_count()}), flush=True)
        return
    if args.mixing_only:
        if args.anderson < 1:
            raise SystemExit("--mixing-only needs --anderson >= 1")
        slice_ms, reduce_ms, mix_ms = pr.time_iterations_mixing(float(gammas[0]), args.mixing_only, opts)
        print(json.dumps({"workload": W["desc"], "iterations": args.mixing_only, "anderson": args.anderson,
                          "gamma_index": 0, "slice_ms": slice_ms, "reduce_ms": reduce_ms, "mix_ms": mix_ms}),
              flush=True)
        return
    if args.iterations_only:
        slice_ms, reduce_ms = pr.time_iterations(float(gammas[len(gammas) // 2]), args.iterations_only, opts)
        print(json.dumps({"workload": W["desc"], "iterations": args.iterations_only, "slice_variant": args.slice_variant,
                          "slice_ms": slice_ms, "reduce_ms": reduce_ms}), flush=True)
        return
    U_dev = torch.empty((G, n, p), dtype=torch.float32, device="cuda")
    L_dev = torch.empty((G, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def step():
        pr.build_knn(W["k"], phi=W.get("phi", 0.0), phi_auto=W.get("phi_auto", False), normalize=W["normalize"])
        pr.reset_path()
        _, _, stats, _ = pr.solve_path(gammas, opts, device=True, U_out=U_dev, labels_out=L_dev)
        return stats

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times, iters = [], []
    stream = torch.cuda.current_stream()
    l0 = ccx.kernel_launches()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.cuda.nvtx.range_push("timed_step")   # lets a profiler select the timed launches
            stats = step()
            torch.cuda.nvtx.range_pop()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(sum(s["iters"] for s in stats))
            per_gamma = [(int(s["iters"]), int(s["converged"]), int(s["n_fused"]), int(s["mixing_iters"]))
                         for s in stats]
            recomputes = int(sum(s["recomputes"] for s in stats))
    launches = ccx.kernel_launches() - l0
    if dist:
        dist.barrier()
    t_step = statistics.median(times)
    edge_updates = m * p * statistics.median(iters)
    t_max = dist_max(t_step, dist)
    total_updates = dist_sum(edge_updates, dist)
    value = total_updates / t_max

    # roofline of the fused node/edge kernel, timed on its own stream
    mid = float(gammas[len(gammas) // 2])
    slice_ms, reduce_ms = pr.time_iterations(mid, 200, opts)
    frac_missing = 0.0 if W["mask"] is None else float(1.0 - W["mask"].mean())
    p4 = (p + 3) // 4 * 4
    # algorithmic bytes of one MM iteration by the method's own accounting
    # (factored V, one projection sweep per iteration): per matrix entry, the
    # RHS gather and node update read X, U, A' and A and write U and R
    # (24 B), the projection sweep reads R and A and writes A (12 B), the edge
    # pass reads A, A' and U (12 B); per edge, s and the CSR entry (12 B) and
    # the new ||b|| (4 B)
    es = 8.0 if prec == ccx.CCX_FP64 else 4.0             # matrix element bytes (the model is per FP32 element)
    alg_bytes = 48.0 * (es / 4.0) * n * p + 16.0 * m
    # this kernel's own minimum traffic: per matrix entry, A (hi, lo) read and
    # written, Delta_{m-1} read, Delta_m written, X read, one mask bit, and
    # (missing entries) two offsets read and written; per edge, the momentum
    # pair (t_m, t_{m-1}) read once for each of its three sweep positions
    own_bytes = (28.0 + 1.0 / 8.0 + 16.0 * frac_missing) * n * p4 + m * 3 * 8
    peaks, peak_src = load_peaks()
    achieved = alg_bytes / (slice_ms * 1e-3) / 1e9
    traffic, traffic_note = stored_traffic(args.workload)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # host buffers in pinned (page-locked) memory, allocated once outside the timed region as a
        # serving process would: the inputs are copied in and U and the labels copied out every step
        Xh = torch.from_numpy(W["X"]).pin_memory().numpy()
        Mh = torch.from_numpy(W["mask"]).pin_memory().numpy() if W["mask"] is not None else None
        Uh = torch.empty((G, n, p), dtype=torch.float32, pin_memory=True).numpy()
        Lh = torch.empty((G, n), dtype=torch.int32, pin_memory=True).numpy()

        def e2e_step():
            q = ccx.Problem(Xh, Mh, prec)
            q.build_knn(W["k"], phi=W.get("phi", 0.0), phi_auto=W.get("phi_auto", False), normalize=W["normalize"])
            _, _, st2, _ = q.solve_path(gammas, opts, U_out=Uh, labels_out=Lh)
            q.close()
            return st2
        # the device arm's warm-up steps already loaded the kernels; each call
        # through host buffers is timed whole (creation included).  Median over
        # the timed steps, at most 5 of them: one step is a whole gamma path
        runs = max(1, min(args.steps, 5))
        tes, upds = [], []
        for _ in range(runs):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st2 = e2e_step()
            torch.cuda.synchronize()
            tes.append(dist_max(time.perf_counter() - t0, dist))
            upds.append(dist_sum(m * p * sum(s["iters"] for s in st2), dist))
        k = int(np.argsort(tes)[len(tes) // 2])
        te, upd = tes[k], upds[k]
        h2d = Xh.nbytes + (Mh.nbytes if Mh is not None else 0)
        d2h = Uh.nbytes + Lh.nbytes
        e2e = {"value": upd / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "seconds_per_step": te, "solves_per_s": ws / te, "runs": runs, "host_memory": "pinned"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, steps_o, el = oracle_sample(W, args.ref_seconds, gammas, (ei, ej, w))
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{steps_o} literal FP64 MM steps (exact projection) of the oracle at the middle gamma, "
                         f"{el:.1f} s, same edges"}
    if rank == 0:
        hbm = peaks.get("hbm_gbs")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == ccx.CCX_FP64 else "f32", "data": "synthetic",
                "config": run_config(W, m, ws),
                "iters_per_step": int(statistics.median(iters)),
                "per_gamma_iters_converged_fused_mixed": per_gamma,
                "anderson": args.anderson,
                "fp64_recomputes_per_step": recomputes,
                "solves_per_s": ws / t_max,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_note,
                             "kernel": "pd_slice_kernel", "slice_ms": slice_ms, "reduce_ms": reduce_ms,
                             "alg_bytes_per_launch": alg_bytes,
                             "alg_bytes_model": "48 n p + 16 |E| (one projection sweep per iteration; doubled "
                                                "per element on the FP64 path)",
                             "own_min_bytes_per_launch": own_bytes,
                             "frac_own_bytes": own_bytes / (slice_ms * 1e-3) / 1e9 / hbm,
                             "target_frac": 0.6,
                             "measured_limiter": "shared-memory gathers of neighbour rows and their latency "
                                                 "(ncu: wavefronts and scoreboard stalls), not DRAM",
                             "peak_source": f"{peak_src} (of measured copy bandwidth)"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
