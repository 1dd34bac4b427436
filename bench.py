#!/usr/bin/env python
"""Benchmark: right-hand sides solved per second to relative residual 1e-6 with
two-level ORAS-preconditioned FGMRES (arXiv 2004.06309), mixed precision versus
FP64, with p50/p99 latency per right-hand side.

Workload (default): the 5 Hz Overthrust-shaped synthetic model -- 20 x 20 x 4.65
km, layered 2-6 km/s with two thrust-fold surfaces and 5% random texture, Q =
100; nested P2 tetrahedral meshes at 5 fine / 2.5 coarse nodes per wavelength
(coarse 63 x 63 x 9 cells x 6 tets, fine its uniform refinement: 2.37M dofs);
64 subdomains, overlap 2, two-level ORAS,
FGMRES(50), one source at (2.5, 2.5, 0.58) km.  A step is one hz_solve of that
right-hand side to 1e-6 (the per-frequency factorisation is done once before the
timed region and reported separately).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hz|reference]

One JSON line on rank 0.  Under torchrun every rank solves its own replica of
the workload (no collective on the data path; replicas only).
"""
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

METRIC = "RHS solved/s to rel. residual 1e-6, mixed vs FP64 ORAS-GMRES; p50/p99 latency"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (non-tensor) nominal, from the platform figures
WORKLOADS = {
    "overthrust-5hz": dict(kind="overthrust", cells=None, freq=5.0, nsub=64, overlap=2,
                           restart=50),
    "overthrust-medium": dict(kind="overthrust", cells=None, freq=2.5, nsub=16, overlap=2,
                              restart=50),
    "overthrust-small": dict(kind="overthrust", cells=None, freq=1.25, nsub=8, overlap=2,
                             restart=50),
    # the batching form: 128 sources on the 16 x 8 surface grid at 50 m depth, uneven parts
    # (weights drawn in [0.6, 1.4]), pseudo-block FGMRES with 16 slots, mixed precision
    "overthrust-5hz-128": dict(kind="overthrust", cells=None, freq=5.0, nsub=64, overlap=2, restart=50,
                               part_jitter=0.4, nrhs=128, block=16, precisions=["mixed"],
                               fp64_note="not run in this workload: the 5 Hz FP64 figure is in overthrust-5hz"),
    # the precision form at 10 Hz: about 15M P2 dofs (1.19 coarse edges per slowest
    # wavelength), 512 subdomains, complex64 local factors with the FP64 outer loop.  Overlap
    # 1, the iterative coarse solve and factorisation in groups of 64 subdomains keep it on
    # one GPU; there is no FP64 arm (its complex128 factors alone would need about 240 GB).
    "overthrust-10hz": dict(kind="overthrust", cells=None, epw=1.19, freq=10.0, nsub=512, overlap=1,
                            restart=50, coarse="oras", coarse_tol=0.1, factor_group=64, precisions=["mixed"],
                            fp64_check_tol=1e-10,
                            fp64_note="not run: the complex128 local factors alone would need about 240 GB"),
    "tiny": dict(kind="tiny"),
}
# Inner iterations each full workload takes to 1e-6 on the GPU path (the 5 Hz count, 74 in both
# precisions, is pinned by the full-size GPU test to 74 +- 2; the 10 Hz count is that of its
# inner coarse tolerance 0.1).  The reference arm runs in its own
# process, before the GPU arm, and carries its samples to the workload with these counts.
FULL_WORKLOAD_ITERATIONS = {"overthrust-5hz": 74, "overthrust-10hz": 176}


def workload_dofs(name):
    """P2 dofs of an Overthrust-shaped workload: (2 nx + 1)(2 ny + 1)(2 nz + 1) on the fine grid."""
    nx, ny, nz = synth_cells(WORKLOADS[name])
    return (4 * nx + 1) * (4 * ny + 1) * (4 * nz + 1)
# kernels of each timed phase (hz_profile)
PHASE_KERNELS = {
    "local_solve": "k_fwd_c64 / k_bwd_partial_c64 (k_fwd / k_bwd_partial_c128 in FP64), one launch per tree level",
    "coarse": "k_spmv_real, coarse sweeps (or the inner GMRES of the iterative coarse solve), k_spmv_real",
    "cgs2": "k_mdot, k_maxpy, k_reduce",
    "spmv": "k_spmv",
}
# DRAM traffic / panel bytes of the complex64 local sweeps (ncu, medium workload, three launches
# each of the forward and backward sweep; an upper bound of traffic / algorithmic bytes)
LOCAL_SWEEP_TRAFFIC_RATIO = 1.054
# Oracle samples for the CPU baseline / reference arm: same generator, 1/240 and 1/43 of the
# 5 Hz workload's dofs.
ORACLE_SAMPLES = {
    "small": dict(kind="overthrust", cells=None, freq=0.625, nsub=8, overlap=2, restart=50),
    "medium": dict(kind="overthrust", cells=None, freq=1.25, nsub=8, overlap=2, restart=50),
}


def clocks_dir(args):
    """Folder for the clock-sample CSV written during the timed region."""
    d = args.clocks_dir or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d


def synth_cells(spec):
    import synth
    return spec["cells"] or synth.overthrust_cells(spec["freq"], spec.get("epw", 1.25))


def make_problem(spec):
    import synth
    if spec["kind"] == "tiny":
        return synth.tiny_problem()
    return synth.overthrust_problem(seed=0, freq=spec["freq"], cells=synth_cells(spec), nsub=spec["nsub"],
                                    overlap=spec["overlap"], restart=spec["restart"], levels=2,
                                    part_jitter=spec.get("part_jitter", 0.0))



def workload_config(args, spec, world, n=None):
    """The bench line's ``config``: the workload as it is defined, so that the GPU arm and the
    reference arm print the same object.  ``n`` (the dof count the library reports) defaults to
    the count the workload's mesh has."""
    if spec["kind"] == "tiny":
        p = make_problem(spec)                       # P1: one dof per vertex
        n0, nsub, overlap, levels, restart, freq = len(p.mesh.xyz), p.nsub, p.overlap, p.levels, p.restart, p.freq
    else:
        nx, ny, nz = synth_cells(spec)
        n0 = (4 * nx + 1) * (4 * ny + 1) * (4 * nz + 1)
        nsub, overlap, levels, restart, freq = spec["nsub"], spec["overlap"], 2, spec["restart"], spec["freq"]
    nrhs = spec["nrhs"] if args.nrhs == 1 and spec.get("nrhs") else args.nrhs
    block = spec["block"] if args.block == 0 and spec.get("block") else args.block
    return {"workload": args.workload, "n_dofs": int(n if n is not None else n0), "nsub": nsub, "overlap": overlap,
            "levels": 2 if levels == 2 else 1, "restart": restart, "tol": 1e-6,
            "rhs_per_step": nrhs, "block_size": block, "freq_hz": freq,
            "part_jitter": spec.get("part_jitter", 0.0),
            "coarse_solver": spec.get("coarse", args.coarse), "recycle": args.recycle,
            "coarse_tol": args.coarse_tol or spec.get("coarse_tol", 0.0),
            "factor_group": spec.get("factor_group", 0), "tune_sweeps": args.tune_sweeps,
            "l2": "inputs larger than L2 (factors >> 129 MB)",
            "parallelism": f"replicas x{world}"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    def __init__(self, index, path):
        self.path = path
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
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
                "samples": len(sm), "reasons": sorted(reasons)}


def run_oracle_sample(name, steps, warmup):
    """Time the FP64 oracle (as it stands) on one bounded sample; one solve per step.  The
    factorisation is excluded; the solve window's wall-clock bounds are returned so that
    concurrent copies can be timed over their common window."""
    from oracle.solver import OracleSolver
    p = make_problem(ORACLE_SAMPLES[name])
    S = OracleSolver(p)
    S.factor()
    b = S.rhs()[:, 0]
    times, its = [], []
    t_first = None
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        if s == warmup:
            t_first = time.time()
        x, it, rel, ok = S.solve(b)
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
            its.append(it)
    return dict(n=S.n, seconds=statistics.mean(times), iterations=int(statistics.median(its)),
                cores=1, times=times, t_start=t_first, t_end=time.time())


def _oracle_cmd(name, steps, warmup):
    return [sys.executable, os.path.abspath(__file__), "--oracle-sample", name, "--steps", str(steps),
            "--warmup", str(warmup)]


_ONE_THREAD = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _last_json(text):
    for line in text.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("oracle sample printed no result")


def oracle_subprocess(name, steps, warmup):
    """One single-threaded oracle process on one sample."""
    env = dict(os.environ, **_ONE_THREAD)
    out = subprocess.run(_oracle_cmd(name, steps, warmup), capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return _last_json(out.stdout)


def oracle_concurrent(name, steps, warmup, nproc):
    """nproc single-threaded oracle processes at once, one per host core: right-hand sides
    solved per second by all of them over their common solve window."""
    env = dict(os.environ, **_ONE_THREAD)
    procs = [subprocess.Popen(_oracle_cmd(name, steps, warmup), stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(nproc)]
    res = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(_last_json(out))
    t0 = min(r["t_start"] for r in res)
    t1 = max(r["t_end"] for r in res)
    return dict(rhs_per_s=sum(len(r["times"]) for r in res) / (t1 - t0), nproc=nproc, n=res[0]["n"],
                iterations=res[0]["iterations"], window_s=t1 - t0)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def oracle_baseline(n_full, it_full, steps, warmup):
    """The FP64 oracle's throughput on the host cores, carried to the full workload.

    - Cost per iteration is measured on two samples of the same generator (0.625 and
      1.25 Hz, 8 subdomains each) and its growth exponent alpha fitted between them
      (t_iter ~ n^alpha; the subdomains' direct solves make alpha > 1); the full workload's
      time per iteration is the larger sample's carried to n_full with that exponent.
    - P concurrent single-threaded copies of the larger sample run on the P host cores
      this process may use (os.sched_getaffinity); their measured aggregate speedup over
      one copy scales the single-process figure.
    The result is right-hand sides per second of the full workload at it_full iterations."""
    import math
    a = oracle_subprocess("small", 1, 1)
    b = oracle_subprocess("medium", 1, 1)
    ta, tb = a["seconds"] / a["iterations"], b["seconds"] / b["iterations"]
    alpha = math.log(tb / ta) / math.log(b["n"] / a["n"])
    t_iter = tb * (n_full / b["n"]) ** alpha
    single = 1.0 / (t_iter * it_full)
    ncores = len(os.sched_getaffinity(0))
    conc = oracle_concurrent("medium", steps, warmup, ncores)
    speedup = conc["rhs_per_s"] * b["seconds"]
    value = single * speedup
    sample = (f"FP64 oracle solves (factorisation excluded) of the same generator: per-iteration cost at "
              f"{a['n']} and {b['n']} dofs (8 subdomains each) fits t ~ n^{alpha:.2f}, carried to {n_full} dofs "
              f"x {it_full} iterations ({single:.3g} RHS/s on one core); {ncores} concurrent single-threaded "
              f"copies of the {b['n']}-dof sample on {cpu_model()} ran {speedup:.1f}x one copy")
    return dict(value=value, cores=ncores, sample=sample, alpha=alpha, single_core=single, speedup=speedup,
                samples={"small": {"n": a["n"], "s_per_iter": ta}, "medium": {"n": b["n"], "s_per_iter": tb}})


def max_over_ranks(x, dist, device):
    """Slowest rank's time: the whole-job figure of a replicas-only run."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, max_seconds):
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    return units_per_rank * world / max_seconds


# Serving workload: the request stream over 3 seeded Overthrust-shaped models and 5
# frequencies, scaled down 2x in frequency (8x in dofs) so that cold-loading all 15
# problems and serving the stream takes about a minute per precision.
SERVE_SEEDS = (0, 1, 2)
SERVE_FREQS = (1.0, 1.25, 1.5, 2.0, 2.5)


def serve_problem(seed, f):
    """A served problem: the seeded model meshed for frequency f like the 5 Hz workload,
    with about 37k dofs per subdomain at and above 4.5 Hz (fewer, larger-share parts below)."""
    import synth
    nsub = 8 if f < 1.5 else (16 if f < 3.0 else (32 if f < 4.5 else 64))
    return synth.overthrust_problem(seed=seed, freq=f, nsub=nsub, overlap=2, restart=50, levels=2)


def serve_requests(rng, nreq, rate, max_batch, nprob):
    """Poisson arrivals (exponential gaps at `rate` per second); each request names a
    problem uniformly, and 1..max_batch sources at uniform surface positions, 50 m deep."""
    import numpy as np
    gaps = rng.exponential(1.0 / rate, nreq)
    out = []
    for k in range(nreq):
        pid = int(rng.integers(0, nprob))
        nb = int(rng.integers(1, max_batch + 1))
        xy = rng.uniform(0.5, 19.5, (nb, 2))
        pts = np.column_stack([xy, np.full(nb, 0.05)])
        out.append((float(gaps[k]), pid, pts))
    return out


def serve_bench(args):
    """Continuous-batching server under a Poisson request stream; p50/p99 request latency
    and RHS/s, mixed precision against FP64."""
    import threading

    import numpy as np
    import torch
    from paper_2004_06309_gb300 import build, hz
    torch.cuda.set_device(0)
    build.build()
    t0 = time.time()
    freqs = tuple(args.serve_freqs) if args.serve_freqs else SERVE_FREQS
    probs = [serve_problem(sd, f) for sd in SERVE_SEEDS for f in freqs]
    t_gen = time.time() - t0
    budget = 150 * 10**9
    res = {}
    for pname in ({"both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.precision]):
        srv = hz.Server(slots=args.serve_slots, precision=hz.HZ_MIXED if pname == "mixed" else hz.HZ_FP64,
                        hbm_budget=budget)
        deadline = time.time() + args.serve_max_s

        def left():
            return max(1.0, deadline - time.time())

        def log(msg):
            print(f"[serve {pname} {time.time() - t0:7.1f} s] {msg}", file=sys.stderr, flush=True)
        ids = [srv.add_problem(p) for p in probs]
        # cold start: one single-source request per problem loads every factorisation
        tc = time.time()
        warm = [srv.submit(i, [[10.0, 10.0, 0.05]], 1e-6) for i in ids]
        for r in warm:
            srv.wait(r, timeout=left())
        t_cold = time.time() - tc
        log(f"cold start of {len(ids)} problems in {t_cold:.1f} s")
        dofs = [srv.ndofs(i) for i in ids]
        # capacity: a closed burst of requests with the stream's batch mix
        rng = np.random.default_rng(11)
        burst = serve_requests(rng, args.serve_burst or max(args.warmup, 3) * 8, 1.0, args.serve_batch, len(probs))
        tb = time.time()
        reqs = [srv.submit(pid, pts, 1e-6) for _, pid, pts in burst]
        for r in reqs:
            srv.wait(r, timeout=left())
        cap = sum(len(p) for _, _, p in burst) / (time.time() - tb)
        log(f"capacity burst: {len(burst)} requests, {cap:.2f} RHS/s")
        rate = 0.7 * cap / ((1 + args.serve_batch) / 2.0)        # ~70 % of the measured capacity
        stream = serve_requests(np.random.default_rng(12), args.steps, rate, args.serve_batch, len(probs))
        s0 = srv.stats()
        clocks = Clocks(0, os.path.join(clocks_dir(args), f"clocks_serve_{pname}.csv"))
        done = []
        lock = threading.Lock()

        def collect(r, n_src, n_dof):
            X, inf, t = srv.wait(r, timeout=left())
            with lock:
                done.append((t["latency_s"], n_src, max(i for i, _, _ in inf), all(st == 0 for _, st, _ in inf),
                             n_src * n_dof * 16))

        threads = []
        ts = time.time()
        nxt = ts
        for gap, pid, pts in stream:
            nxt += gap
            dt = nxt - time.time()
            if dt > 0:
                time.sleep(dt)
            r = srv.submit(pid, pts, 1e-6)
            th = threading.Thread(target=collect, args=(r, len(pts), dofs[pid]))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        wall = time.time() - ts
        ck = clocks.stop()
        s1 = srv.stats()
        lat = np.array([d[0] for d in done])
        nrhs = sum(d[1] for d in done)
        res[pname] = dict(rhs_per_s=nrhs / wall, p50=float(np.percentile(lat, 50, method="inverted_cdf")),
                          p99=float(np.percentile(lat, 99, method="inverted_cdf")), requests=len(done), rhs=nrhs,
                          all_ok=all(d[3] for d in done), max_iterations=max(d[2] for d in done),
                          capacity_rhs_per_s=cap, rate_req_per_s=rate, cold_start_s=t_cold,
                          factor_seconds=s1["factor_seconds"], factorisations=s1["factorisations"],
                          evictions=s1["evictions"], peak_resident_gb=s1["peak_resident_bytes"] / 1e9,
                          launches=s1["launches"] - s0["launches"], clocks=ck, wall_s=wall, dofs=dofs,
                          h2d_bytes_per_request=sum(24 * d[1] for d in done) / len(done),
                          d2h_bytes_per_request=sum(d[4] for d in done) / len(done))
        srv.close()
        torch.cuda.empty_cache()
    main_p = "mixed" if "mixed" in res else "fp64"
    R = res[main_p]
    line = {
        "metric": METRIC, "value": R["rhs_per_s"], "unit": "RHS/s", "n_gpus": 1, "steps": R["requests"],
        "warmup": len(probs), "ms_per_step": 1e3 * R["wall_s"] / max(R["requests"], 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "complex64 subdomain factors/solves + complex128 Krylov, SpMV, coarse" if main_p == "mixed"
        else "complex128",
        "data": "synthetic",
        "config": {"workload": "serving: Poisson stream over 3 Overthrust-shaped models x 5 frequencies",
                   "seeds": list(SERVE_SEEDS), "freqs_hz": list(freqs),
                   "dofs": R["dofs"],
                   "batch_sources": [1, args.serve_batch], "slots": args.serve_slots, "hbm_budget_gb": budget / 1e9,
                   "tol": 1e-6, "arrival": "Poisson at 70% of the measured closed-loop capacity",
                   "l2": "factors and Krylov bases >> 129 MB", "parallelism": "replicas x1"},
        "latency_ms": {"p50": 1e3 * R["p50"], "p99": 1e3 * R["p99"]},
        "e2e": {"value": R["rhs_per_s"], "unit": "RHS/s", "h2d_bytes_per_step": R["h2d_bytes_per_request"],
                "d2h_bytes_per_step": R["d2h_bytes_per_request"],
                "note": "value is already end to end (host wall clock from submission of host source "
                        "coordinates to collection of host solutions); a step is one request"},
        "gpu_launches": R["launches"], "clocks": R["clocks"], "serving": R,
        "generate_seconds": t_gen,
    }
    if "fp64" in res and main_p != "fp64":
        line["fp64"] = res["fp64"]
    print(json.dumps(line))


def trends_bench(args):
    """Shape of the paper's Table 1 and its remarks on synthetic models (no real model):
    iterations of one- and two-level ORAS-FGMRES against frequency (mesh and subdomain
    count growing with it), the effect of attenuation Q, and the cost of 10 right-hand
    sides against one.  Mixed precision, tol 1e-6, one source at (2.5, 2.5, 0.58) km."""
    import numpy as np
    import torch
    import synth
    from paper_2004_06309_gb300 import build, hz
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def run(p, levels, nrhs=1, block=0):
        G = hz.Solver(p, precision=hz.HZ_MIXED, stream=stream, block_size=block)
        G.factor()
        if nrhs > 1:
            B = torch.from_numpy(np.asfortranarray(G.point_sources(synth.surface_source_grid()[:nrhs]))).cuda()
        else:
            B = torch.from_numpy(G.point_sources(p.sources)[:, 0].copy()).cuda()
        G.solve(B)                                   # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        X, info = G.solve(B)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        n = G.n
        G.close()
        torch.cuda.empty_cache()
        return dict(n=n, iterations=max(i[0] for i in info), seconds=dt, ok=all(i[1] == 0 for i in info))

    # the paper's resolution (coarse edges of 1/2.5 of the wavelength) at three frequencies,
    # then the 5 Hz workload's own mesh (half that resolution)
    rows = [(0.625, 2.5, 8), (1.25, 2.5, 16), (2.5, 2.5, 64), (5.0, 1.25, 64)]
    table = []
    for f, epw, nsub in rows:
        cells = synth.overthrust_cells(f, epw)
        row = {"freq_hz": f, "coarse_elems_per_wavelength": epw, "cells": list(cells), "nsub": nsub}
        for lv in (1, 2):
            p = synth.overthrust_problem(seed=0, freq=f, cells=cells, nsub=nsub, overlap=2, levels=lv)
            r = run(p, lv)
            row["n_dofs"] = r["n"]
            row[f"{lv}level"] = {"iterations": r["iterations"], "seconds": r["seconds"], "ok": r["ok"]}
        table.append(row)
    qrows = []
    for Q in (50.0, 100.0, 1000.0):
        p = synth.overthrust_problem(seed=0, freq=1.25, cells=synth.overthrust_cells(1.25, 2.5), nsub=16,
                                     overlap=2, levels=2, Q=Q)
        r = run(p, 2)
        qrows.append({"Q": Q, "iterations": r["iterations"], "ok": r["ok"]})
    p = synth.overthrust_problem(seed=0, freq=5.0, nsub=64, overlap=2, levels=2)
    one = run(p, 2)
    ten = run(p, 2, nrhs=10, block=16)
    line = {"experiment": "trends (Table 1 shape on synthetic Overthrust-shaped models)",
            "iterations_vs_frequency": table, "attenuation_1p25hz_paper_resolution": qrows,
            "multi_rhs_5hz": {"one_rhs_s": one["seconds"], "ten_rhs_s": ten["seconds"],
                              "ratio_10_to_1": ten["seconds"] / one["seconds"],
                              "iterations": [one["iterations"], ten["iterations"]]},
            "precision": "mixed", "tol": 1e-6}
    print(json.dumps(line))


def crossover_bench(args):
    """One level against two on the 5 Hz workload's mesh (coarse (63, 63, 9) cells, 2.37M
    P2 dofs, 64 subdomains) at four frequencies, i.e. at 1.25, 1.5, 2 and 2.5 coarse element
    edges per slowest wavelength (2.5, 3, 4 and 5 fine P2 elements): where the coarse space
    starts to pay.  Mixed precision, tol 1e-6, one source at (2.5, 2.5, 0.58) km; one
    warm-up and one timed solve per row."""
    import torch
    import synth
    from paper_2004_06309_gb300 import build, hz
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cells = synth.overthrust_cells(5.0, 1.25)
    rows = []
    for epw in (1.25, 1.5, 2.0, 2.5):
        f = 5.0 * 1.25 / epw
        row = {"coarse_elems_per_wavelength": epw, "fine_elems_per_wavelength": 2 * epw, "freq_hz": f,
               "cells": list(cells)}
        for lv in (1, 2):
            p = synth.overthrust_problem(seed=0, freq=f, cells=cells, nsub=64, overlap=2, levels=lv)
            G = hz.Solver(p, precision=hz.HZ_MIXED, stream=stream)
            G.factor()
            b = torch.from_numpy(G.point_sources(p.sources)[:, 0].copy()).cuda()
            G.solve(b)
            torch.cuda.synchronize()
            t = time.perf_counter()
            x, info = G.solve(b)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            row["n_dofs"] = G.n
            row[f"{lv}level"] = {"iterations": info[0][0], "seconds": dt, "rhs_per_s": 1.0 / dt,
                                 "ok": info[0][1] == 0}
            G.close()
            torch.cuda.empty_cache()
        rows.append(row)
    print(json.dumps({"experiment": "one level against two on the 5 Hz mesh", "rows": rows,
                      "precision": "mixed", "tol": 1e-6}))


def block_bench(args):
    """Block FGMRES against pseudo-block FGMRES on the 5 Hz workload: 16 sources from the
    16 x 8 surface grid at 50 m depth, solved with block sizes 4, 8 and 16 (16 / S batches
    of one block Krylov space each, against 16 / S rounds of S independent slots), mixed
    precision, tol 1e-6.  With --recycle k a third row per block size runs block GCRO-DR
    (the block batches share a recycled space of dimension k).  One warm-up solve of S other
    sources of the grid, then one timed solve of the 16 sources per configuration."""
    import numpy as np
    import torch
    import synth
    from paper_2004_06309_gb300 import build, hz
    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = make_problem(WORKLOADS["overthrust-5hz"])
    grid = synth.surface_source_grid()
    rows = []
    kinds = ("pseudo", "block") + (("block-gcrodr",) if args.recycle else ())
    for S in args.block_sizes:
        for kind in kinds:
            G = hz.Solver(p, precision=hz.HZ_MIXED, stream=stream, block_size=S,
                          krylov=hz.HZ_KRYLOV_PSEUDO_BLOCK if kind == "pseudo" else hz.HZ_KRYLOV_BLOCK,
                          recycle=args.recycle if kind == "block-gcrodr" else 0)
            G.factor()
            B = torch.from_numpy(np.asfortranarray(G.point_sources(grid[:16]))).cuda()
            W = torch.from_numpy(np.asfortranarray(G.point_sources(grid[16:16 + S]))).cuda()
            G.solve(W)
            torch.cuda.synchronize()
            t = time.perf_counter()
            X, info = G.solve(B)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            rows.append({"block_size": S, "krylov": kind, "rhs_per_s": 16 / dt, "seconds": dt,
                         "iterations": [int(i[0]) for i in info], "ok": all(i[1] == 0 for i in info),
                         "max_rel_residual": max(i[2] for i in info)})
            if kind == "block-gcrodr":
                rows[-1]["recycle"] = args.recycle
            G.close()
            torch.cuda.empty_cache()
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"experiment": "block FGMRES against pseudo-block FGMRES, 5 Hz workload, 16 sources",
                      "rows": rows, "precision": "mixed", "tol": 1e-6}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hz", choices=["hz", "reference"])
    ap.add_argument("--workload", default="overthrust-5hz",
                    choices=list(WORKLOADS) + ["serving", "trends", "crossover", "block"])
    ap.add_argument("--serve-batch", type=int, default=16, help="largest sources per request (serving)")
    ap.add_argument("--serve-freqs", type=float, nargs="+", default=None,
                    help="frequencies of the served problems (default: 1.0 1.25 1.5 2.0 2.5)")
    ap.add_argument("--serve-slots", type=int, default=16, help="slots per served problem")
    ap.add_argument("--serve-max-s", type=float, default=1500.0,
                    help="wall-clock limit of the serving run; a request still open then raises")
    ap.add_argument("--serve-burst", type=int, default=0,
                    help="requests of the closed capacity burst (0: 8 x max(warmup, 3))")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default="",
                    help="folder for the nvidia-smi clock samples of the timed region (default: system temp)")
    ap.add_argument("--block", type=int, default=0,
                    help="pseudo-block FGMRES block size (right-hand sides sharing each operator application)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="right-hand sides per step (sources from the 16 x 8 surface grid at 50 m depth)")
    ap.add_argument("--leaf", type=int, default=0, help="nested-dissection leaf size (0: library default)")
    ap.add_argument("--maxsn", type=int, default=0, help="widest supernode (0: library default)")
    ap.add_argument("--coarse", default="direct", choices=["direct", "oras"],
                    help="coarse solve: direct LDL^T of E, or inner GMRES with coarse one-level ORAS")
    ap.add_argument("--coarse-tol", type=float, default=0.0, help="inner coarse tolerance (0: library default)")
    ap.add_argument("--coarse-maxit", type=int, default=0, help="inner coarse iterations at most (0: default)")
    ap.add_argument("--recycle", type=int, default=0,
                    help="GCRO-DR: recycled-space dimension kept across the step's right-hand sides (0: FGMRES)")
    ap.add_argument("--tune-sweeps", type=int, default=1,
                    help="1: autotune the sweep task shapes at the first factorisation (0: library default shapes)")
    ap.add_argument("--block-sizes", type=int, nargs="+", default=[4, 8, 16],
                    help="block sizes of the block-against-pseudo-block comparison (--workload block)")
    ap.add_argument("--one-level-steps", type=int, default=3,
                    help="timed steps of the one-level arm on the same mesh (mixed precision; 0: skip)")
    ap.add_argument("--oracle-sample", default="", help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.oracle_sample:
        print(json.dumps(run_oracle_sample(args.oracle_sample, args.steps, args.warmup)))
        return

    if args.workload in ("serving", "trends", "crossover", "block") and args.impl == "hz":
        if int(os.environ.get("RANK", "0")) == 0:
            {"serving": serve_bench, "trends": trends_bench, "crossover": crossover_bench,
             "block": block_bench}[args.workload](args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        full_it = FULL_WORKLOAD_ITERATIONS.get(args.workload)
        if full_it is None:                            # sample-sized workloads: the oracle solves them
            samp = oracle_subprocess("medium", args.steps, args.warmup)
            base = dict(value=1.0 / samp["seconds"], cores=1, sample="the FP64 oracle on the medium sample itself")
        else:
            base = oracle_baseline(workload_dofs(args.workload), full_it, args.steps, args.warmup)
        val = base["value"]
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "RHS/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / val,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "complex128",
                "data": "synthetic", "config": workload_config(args, WORKLOADS[args.workload], world),
                "cpu_baseline": {"value": val, "unit": "RHS/s", "cores": base["cores"], "kind": "oracle",
                                 "sample": base["sample"]},
                "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import numpy as np
    import torch

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)

    from paper_2004_06309_gb300 import build, hz
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()

    spec = WORKLOADS[args.workload]
    if args.nrhs == 1 and spec.get("nrhs"):
        args.nrhs = spec["nrhs"]
    if args.block == 0 and spec.get("block"):
        args.block = spec["block"]
    t0 = time.time()
    prob = make_problem(spec)
    t_gen = time.time() - t0

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def maxall(x):
        return max_over_ranks(x, dist, "cuda") if dist else x

    precs = {"both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.precision]
    precs = [q for q in precs if q in spec.get("precisions", precs)]
    coarse = spec.get("coarse", args.coarse)
    results = {}
    # a dedicated (non-default) stream, so that the library can capture its iterations as CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    for pname in precs:
        G = hz.Solver(prob, precision=hz.HZ_MIXED if pname == "mixed" else hz.HZ_FP64, stream=stream,
                      leaf_size=args.leaf, max_snode=args.maxsn, block_size=args.block,
                      coarse_solver=hz.HZ_COARSE_ORAS if coarse == "oras" else hz.HZ_COARSE_DIRECT,
                      coarse_tol=args.coarse_tol or spec.get("coarse_tol", 0.0), coarse_maxit=args.coarse_maxit,
                      recycle=args.recycle,
                      factor_group=spec.get("factor_group", 0), tune_sweeps=args.tune_sweeps)
        tf = time.time()
        G.factor()
        torch.cuda.synchronize()
        t_factor = time.time() - tf
        if args.nrhs > 1:
            import synth
            srcs = synth.surface_source_grid()[: args.nrhs]
            b_host = np.asfortranarray(G.point_sources(srcs))
        else:
            b_host = G.point_sources(prob.sources)[:, 0].copy()
        b_dev = torch.from_numpy(b_host).cuda()
        for _ in range(args.warmup):
            x, info = G.solve(b_dev)
        st0 = G.stats()["launches"]
        clocks = Clocks(local, os.path.join(clocks_dir(args), f"clocks_{pname}_r{rank}.csv"))
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        its = []
        for s in range(args.steps):
            x, info = G.solve(b_dev)
            ev[s + 1].record(stream)
            its.append(max(i[0] for i in info))
        barrier()
        ck = clocks.stop()
        launches = G.stats()["launches"] - st0
        step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
        total_ms = maxall(sum(step_ms))
        rel = info[0][2]
        # end to end through the C ABI with host buffers (copies inside the timed region)
        barrier()
        te = time.perf_counter()
        for s in range(args.steps):
            xh, infoh = G.solve(b_host)
        torch.cuda.synchronize()
        e2e_s = maxall(time.perf_counter() - te)
        check = None
        if spec.get("fp64_check_tol") and args.nrhs == 1:
            # no FP64 factors fit: the FP64 outer FGMRES driven to a tight tolerance gives the
            # FP64 solution (to kappa * tol), against which the timed solution's error is taken
            xr, infor = G.solve(b_dev, tol=spec["fp64_check_tol"])
            x1 = x.reshape(-1)
            check = {"reference": f"same context solved to {spec['fp64_check_tol']:g} (FP64 outer FGMRES)",
                     "reference_iterations": infor[0][0], "reference_rel_residual": infor[0][2],
                     "rel_l2_vs_reference": float(torch.linalg.norm(x1 - xr.reshape(-1)) /
                                                  torch.linalg.norm(xr.reshape(-1)))}
        prof = G.profile(reps=3)
        stats = G.stats()
        results[pname] = dict(total_ms=total_ms, step_ms=step_ms, iterations=its, rel=rel, clocks=ck,
                              launches=launches, e2e_s=e2e_s, profile=prof, stats=stats,
                              t_factor=t_factor, n=G.n, check=check)
        G.close()
        del G
        torch.cuda.empty_cache()

    # one-level arm (Eq. 4 alone) on the same mesh and partition, mixed precision: shows
    # where the coarse space pays and where it does not (its resolution, not the method)
    one = None
    if (args.one_level_steps > 0 and prob.levels == 2 and "mixed" in precs and args.nrhs == 1
            and args.workload == "overthrust-5hz"):
        import dataclasses
        p1 = dataclasses.replace(prob, levels=1, coarse=None, fine_parent=None)
        G = hz.Solver(p1, precision=hz.HZ_MIXED, stream=stream, leaf_size=args.leaf, max_snode=args.maxsn)
        tf = time.time()
        G.factor()
        torch.cuda.synchronize()
        t_factor1 = time.time() - tf
        b1 = torch.from_numpy(G.point_sources(prob.sources)[:, 0].copy()).cuda()
        for _ in range(min(args.warmup, 2)):
            G.solve(b1)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.one_level_steps + 1)]
        ev[0].record(stream)
        its1 = []
        for s in range(args.one_level_steps):
            x1, info1 = G.solve(b1)
            ev[s + 1].record(stream)
            its1.append(info1[0][0])
        barrier()
        ms1 = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.one_level_steps)]
        tot1 = maxall(sum(ms1))
        one = dict(value=world * args.one_level_steps / (tot1 / 1e3), ms_per_step=tot1 / args.one_level_steps,
                   iterations=its1[-1], rel_residual=info1[0][2], factor_seconds=t_factor1,
                   latency_ms={"p50": float(np.percentile(ms1, 50)), "p99": float(np.percentile(ms1, 99))})
        G.close()
        del G
        torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    main_p = "mixed" if "mixed" in results else "fp64"
    R = results[main_p]
    n = R["n"]
    K = args.steps
    value = job_throughput(K * args.nrhs, world, R["total_ms"] / 1e3)

    def lat(r):
        s = sorted(r["step_ms"])
        return {"p50": float(np.percentile(s, 50)), "p99": float(np.percentile(s, 99))}

    # roofline of the dominant phase of one iteration
    hbm_peak, peak_kind = load_peaks()
    prof = R["profile"]
    cand = ["spmv", "coarse", "restrict", "local_solve", "prolong", "cgs2"]
    dom = max(cand, key=lambda k: prof[k]["ms"])
    ph = prof[dom]
    # FP64 arithmetic: every phase of the FP64 path; in the mixed path all but the local
    # solves and, with the iterative coarse solve, its complex64 coarse subdomain sweeps
    fp64_phase = main_p == "fp64" or (dom != "local_solve" and not (dom == "coarse" and coarse == "oras"))
    t_s = ph["ms"] / 1e3
    gbs = ph["bytes"] / t_s / 1e9
    tfl = ph["flops"] / t_s / 1e12
    if fp64_phase and ph["flops"] / (FP64_PEAK_TFLOPS * 1e12) > ph["bytes"] / (hbm_peak * 1e9):
        roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 nominal (platform figure)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": None, "peak_source": f"{peak_kind} hbm_gbs (copy)"}
    # the phase's kernels (one launch per tree level and direction for the local solve):
    # its time and launches per run, not one kernel's
    roof.update({"kernel": f"{dom} phase ({main_p}): {PHASE_KERNELS.get(dom, dom)}", "phase_ms_per_run": ph["ms"],
                 "algorithmic_bytes": ph["bytes"], "flops": ph["flops"], "phase_launches_per_run": ph["launches"]})
    roof["local_solve_frac"] = prof["local_solve"]["bytes"] / (prof["local_solve"]["ms"] / 1e3) / 1e9 / hbm_peak
    if dom == "local_solve" and main_p == "mixed":
        # DRAM bytes per run of the complex64 sweeps: ncu (dram__bytes_read/write) on the
        # medium workload measured 1.054 x the panel bytes; the traffic grows with the panel
        # entries, so it is scaled to this workload
        roof["traffic"] = LOCAL_SWEEP_TRAFFIC_RATIO * ph["bytes"]
        roof["traffic_source"] = "ncu dram bytes on overthrust-medium, scaled by algorithmic bytes"

    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": R["total_ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "complex64 subdomain factors/solves + complex128 Krylov, SpMV, coarse" if main_p == "mixed"
        else "complex128",
        "data": "synthetic",
        "config": workload_config(args, spec, world, n),
        "iterations": R["iterations"][-1], "rel_residual": R["rel"],
        "latency_ms": lat(R),
        "factor_seconds": R["t_factor"],
        "e2e": {"value": world * K * args.nrhs / R["e2e_s"], "unit": "RHS/s",
                "h2d_bytes_per_step": n * 16 * args.nrhs, "d2h_bytes_per_step": n * 16 * args.nrhs},
        "gpu_launches": R["launches"],
        "clocks": R["clocks"],
        "roofline": roof,
        "phases_ms": {k: round(v["ms"], 4) for k, v in prof.items()},
        "phases_gbytes": {k: round(v["bytes"] / 1e9, 4) for k, v in prof.items()},
        "phases_gflops": {k: round(v["flops"] / 1e9, 4) for k, v in prof.items()},
        "stats": {k: R["stats"][k] for k in ("nnz", "n_coarse", "sum_ni", "nnz_factor", "nnz_factor_coarse",
                                             "sweep_chunk", "sweep_scale",
                                             "nsupernodes", "nlevels", "front_bytes", "device_bytes",
                                             "setup_seconds", "coarse_solves", "coarse_iterations")},
        "generate_seconds": t_gen,
    }
    if "fp64" in results and main_p != "fp64":
        F = results["fp64"]
        line["fp64"] = {"value": world * K * args.nrhs / (F["total_ms"] / 1e3), "ms_per_step": F["total_ms"] / K,
                        "iterations": F["iterations"][-1], "rel_residual": F["rel"], "latency_ms": lat(F),
                        "factor_seconds": F["t_factor"],
                        "e2e_value": world * K * args.nrhs / F["e2e_s"],
                        "phases_ms": {k: round(v["ms"], 4) for k, v in F["profile"].items()},
                        "phases_gflops": {k: round(v["flops"] / 1e9, 4) for k, v in F["profile"].items()},
                        "clocks": F["clocks"]}
    if R.get("check"):
        line["fp64_check"] = R["check"]
    if "fp64" not in results and spec.get("fp64_note"):
        line["fp64"] = {"value": None, "note": spec["fp64_note"]}
    if one is not None:
        line["one_level"] = dict(one, precision="mixed",
                                 note="levels=1 on the same mesh and partition; no coarse space")
    if not args.no_cpu_baseline and world == 1:
        try:
            if args.workload == "tiny":
                samp = oracle_subprocess("medium", 1, 1)
                base = dict(value=1.0 / samp["seconds"], cores=1, sample="the FP64 oracle on the medium sample")
            else:                                  # this run's own iteration count
                base = oracle_baseline(n, R["iterations"][-1], 3, 1)
            line["cpu_baseline"] = {"value": base["value"], "unit": "RHS/s", "cores": base["cores"],
                                    "kind": "oracle", "sample": base["sample"]}
            for key in ("alpha", "single_core", "speedup"):
                if key in base:
                    line["cpu_baseline"][key] = base[key]
        except Exception as e:  # the GPU line still stands
            line["cpu_baseline"] = {"value": None, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e}"[:300]}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
