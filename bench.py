"""Benchmark of the butterfly hot path on one GB300 (or N independent replicas).

Workload (the precision configuration at full size): the 2D Helmholtz kernel
exp(-i k r)/r between two parallel unit segments at distance 1, n = m = 16384
points, 8 points per wavelength, entries from the kernel's closed form
(formed once per factorization into complex64 entry images of A and A^H, then
streamed by every sketch), leaf 16 (L = 10), tol 1e-6, p = 2, r0 = 16, seed 0.

One step = one pass of the whole hot path: bf_factor (sketch RNG, sketch
products, adaptive leaf bases, peeling, batched QR, B least squares) in the
mixed form -- complex64 sketches and peeling on the tensor cores, pivoted QR,
truncation and the B least squares in FP64 -- then bf_apply of 64
right-hand sides and the sketch error of Sec. 7.  `value` is the factor time
in seconds (device-timed with CUDA events on the launching stream, L2 flushed
before every step by writing a 512 MB buffer); the line also reports the
plain FP64 factor time, the float-float-QR variant, apply GB/s, the roofline
of the dominant kernel and the FP64 oracle timed on the host at the same size.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 16384
LEAF = 16
TOL = 1e-6
NRHS = 64
# initial rank guess of the adaptive leaf loops: the leaf size, so each loop
# ends after one pass (a sketch pass costs the same for any width up to 48
# columns on the tensor-core path; the ranks are still found by the
# truncated QR, Alg. 2)
R0 = 16
# FP32/ALU operations of one 2-D kernel entry in the mixed path, counted from
# its source: float-float differences 16, squares 8, sum 8, rsqrt + Newton 5,
# float-float square-root correction 8, phase 4, pi/2 reduction 5,
# polynomial sin/cos 9, quadrant 6, scaling 2
ALU_OPS_PER_ENTRY = 71
# DRAM bytes (read + write) of one sketch_img_kernel<48> launch at n = 8192
# (the image profile case), from ncu; the image read once, X and Y.  Valid
# only for the kernel source it was captured on (SHA-256 prefix below); after
# any change to that file the line reports traffic null until a new capture.
IMG_TRAFFIC_N8192 = 541691392 + 6283008
IMG_TRAFFIC_SOURCE_SHA = "729e94c36183ee54"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", "0"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def img_traffic_valid() -> bool:
    """Whether the image kernel's source is the one the DRAM traffic was
    captured on."""
    import hashlib
    src = os.path.join(ROOT, "paper_2002_03400_gb300", "csrc", "k_sketch_tc.cu")
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16] == IMG_TRAFFIC_SOURCE_SHA


def oracle_factor_seconds(n: int = N) -> float:
    """Wall time of one oracle factorization (plain FP64 numpy, as it stands)
    of the benchmark workload at n points: Alg. 2 with the kernel formed on
    the fly by the oracle's black box, the same leaf, tol, p and r0."""
    from oracle import butterfly as ob
    from oracle import operators as oo
    from paper_2002_03400_gb300 import inputs
    g = inputs.line_pair(n)
    op = oo.KernelOp(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    L = inputs.leaf_levels(n, LEAF)
    t0 = time.perf_counter()
    ob.factor(op, g.src, g.tgt, L, TOL, 2, R0, seed=0)
    return time.perf_counter() - t0


def bench_config(n: int = N) -> dict:
    """The workload both arms report (identical dicts at the default size)."""
    from paper_2002_03400_gb300 import inputs
    return {"workload": f"helmholtz2d_line_pair_n{n}_kernel", "n": n, "m": n, "leaf": LEAF,
            "L": inputs.leaf_levels(n, LEAF), "tol": TOL, "p": 2, "r0": R0, "seed": 0, "nrhs": NRHS,
            "l2": "flushed (512 MB write) before every step"}


ORACLE_CORES_NOTE = ("numpy FP64 oracle: its GEMMs use the BLAS thread pool (all cores), its kernel-entry "
                     "evaluation one thread")


def profile_case(args):
    """Small cases of one kernel family, sized for ncu captures (a few GB on
    the device at most): the on-the-fly sketch product (n = 8192, 22
    columns, all rows against all sources), the apply of a factorization
    (n = 16384, 64 and 1 right-hand sides, grouped engine then stage
    launches), one factorization (its QR levels) or
    factorizations at n = 8192 with entry images."""
    import torch
    from paper_2002_03400_gb300 import api, inputs
    api.set_sketch_engine(args.engine)
    if args.profile_case == "sketch":
        n = 8192
        g = inputs.line_pair(n)
        plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, precision="mixed")
        op = api.Operator.kernel(plan)
        X = api.colmajor(torch.from_numpy(inputs.random_rhs(n, 22, seed=3)).to(torch.complex64).cuda())
        for _ in range(3):
            op.apply(X)
    elif args.profile_case == "image":
        # three mixed factorizations at n = 8192 with entry images (two
        # 0.8 GB images per factorization): the image kernel and the
        # image-fed sketch products
        n = 8192
        g = inputs.line_pair(n)
        plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                        precision="mixed", r0=R0)
        op = api.Operator.kernel(plan)
        for _ in range(3):
            api.Factorization.factor(plan, op)
    elif args.profile_case == "step":
        # the bench step (mixed factorization, apply of 64 right-hand sides,
        # sketch error), once per --steps
        g = inputs.line_pair(N)
        plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                        precision="mixed", r0=R0)
        op = api.Operator.kernel(plan)
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(N, NRHS, seed=1)).to(torch.complex64).cuda())
        for _ in range(args.steps):
            F = api.Factorization.factor(plan, op)
            F.apply(x)
            F.error(op, 16, seed=7, dtype=x.dtype)
    else:
        g = inputs.line_pair(N)
        plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                        precision="mixed", r0=R0, qr_fp64=True)
        F = api.Factorization.factor(plan, api.Operator.kernel(plan))
        if args.profile_case == "apply":
            # applies of 64 and of 1 complex64 right-hand sides, grouped
            # engine (untuned depth) then stage launches, each engine warmed
            # first; only the applies run between cudaProfilerStart and Stop
            # (ncu --profile-from-start off captures them alone)
            x = api.colmajor(torch.from_numpy(inputs.random_rhs(N, NRHS, seed=1)).to(torch.complex64).cuda())
            x1 = api.colmajor(x[:, :1].clone())
            for eng in ("grouped", "stages"):
                api.set_apply_engine(eng)
                F.apply(x)
                F.apply(x1)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            for eng in ("grouped", "stages"):
                api.set_apply_engine(eng)
                for _ in range(3):
                    F.apply(x)
                for _ in range(3):
                    F.apply(x1)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            api.set_apply_engine("auto")
    torch.cuda.synchronize()
    print("profile case done")


def serving_measure(seconds: float = 4.0, saturation_requests: int = 200):
    """Serving (continuous batching over resident factorizations: arcs n =
    4096 and 16384, caps n = 4096 and 16384; mixed precision, FP64 QR).

    * capacity of the served form: `saturation_requests` requests of the
      serving mix (80% applies of 1..64 complex64/complex128 right-hand
      sides, 20% factor requests n in {4096, 16384, 65536} on arcs/caps) all
      queued at once; requests, applies and factorizations per second over
      the makespan, with the latency percentiles of that backlog;
    * Poisson arrivals at 0.5x and 2x the capacity of a one-request-at-a-
      time plain FP64 baseline (FP64 factors, complex128 products), served
      and baseline replays of the same trace; factor sizes there are 4096
      and 16384 (an FP64 factorization at n = 65536 takes tens of seconds,
      too long for a bounded run)."""
    import torch
    from paper_2002_03400_gb300 import inputs, serve
    sizes = {"arc4k": (4096, "arc"), "arc16k": (16384, "arc"), "cap4k": (4096, "cap"), "cap16k": (16384, "cap")}
    res = {k: serve.build_factor(serve.factor_spec(n, geo, seed=i)) for i, (k, (n, geo)) in enumerate(sizes.items())}
    names = list(res)
    nof = {k: sizes[k][0] for k in res}
    out = {"resident": {k: sizes[k][0] for k in sizes}}

    # capacity of the served form: the whole backlog at t = 0
    # (unit rate: about 1.5 x saturation_requests arrivals, the first kept)
    tr = inputs.serving_trace(1.5 * saturation_requests + 50, 1.0, seed=31, resident=len(names),
                              factor_sizes=(4096, 16384, 65536))[:saturation_requests]
    jobs = serve.make_jobs(tr, names, nof, seed=9)
    for j in jobs:
        j.t_arrive = 0.0
    srv = serve.Server(mem_cap=150e9, factor_workers=2)
    for k, F in res.items():
        srv.add_resident(k, F)
    t0 = time.perf_counter()
    done = srv.run(jobs, realtime=False)
    torch.cuda.synchronize()
    span = time.perf_counter() - t0
    srv.close()
    for j in done:   # new factorizations are not kept
        if j.kind == "factor" and j.result is not None:
            j.result.free()
            j.result = None
    out["capacity"] = dict(serve.throughput_stats(done, span), **{"backlog": serve.latency_stats(done)})

    def baseline(jobs):
        """one request at a time, FP64 factors and complex128 products"""
        t0 = time.perf_counter()
        for j in jobs:
            while time.perf_counter() - t0 < j.t_arrive:
                time.sleep(0.0002)
            if j.kind == "apply":
                x = torch.from_numpy(j.x.astype(np.complex128)).cuda()
                j.result = res[j.target].apply(x).cpu().numpy()
            else:
                spec = dict(j.spec, precision="fp64")
                j.result = serve.build_factor(spec)
                j.result.free()
            torch.cuda.synchronize()
            j.t_done = time.perf_counter() - t0
        return jobs

    # capacity of the baseline: mean service time on a short sample
    probe = serve.make_jobs(inputs.serving_trace(1.0, 40.0, seed=11, resident=len(names), factor_sizes=(4096, 16384)),
                            names, nof, seed=5)
    for j in probe:
        j.t_arrive = 0.0
    t0 = time.perf_counter()
    baseline(probe)
    cap = len(probe) / (time.perf_counter() - t0)
    out["baseline_capacity_req_per_s"] = cap
    out["seconds"] = seconds
    for mult in (0.5, 2.0):
        rate = cap * mult
        tr = inputs.serving_trace(seconds, rate, seed=21, resident=len(names), factor_sizes=(4096, 16384))
        jobs = serve.make_jobs(tr, names, nof, seed=6)
        srv = serve.Server(mem_cap=150e9, factor_workers=2)
        for k, F in res.items():
            srv.add_resident(k, F)
        done = srv.run(jobs, realtime=True)
        srv.close()
        bjobs = baseline(serve.make_jobs(tr, names, nof, seed=6))
        out[f"rate_{mult}x"] = {"rate_req_per_s": rate, "requests": len(jobs),
                                "served": serve.latency_stats(done), "baseline": serve.latency_stats(bjobs)}
    return out


def batched_measure(count: int = 64, reps: int = 2):
    """Batched workload: `count` operators between two separated circular arcs
    (radius 1, opening angles U[30, 90] degrees, centre distance 3, 4-16
    points per wavelength), n drawn from {1024, 2048, 4096, 8192}, leaf 32,
    tol 1e-5, complex64 sketches with FP64 QR: bf_factor_batch (one launch per
    kernel per phase for all operators) against one bf_factor after another,
    wall time of the whole set (device synchronised), plus the sketch error
    of every operator against its bound."""
    import torch
    from paper_2002_03400_gb300 import api, inputs
    sizes = inputs.batched_sizes(count)
    plans = []
    for i, n in enumerate(sizes):
        g = inputs.arc_pair(n, seed=100 + i)
        plans.append(api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=1e-5,
                              precision="mixed", seed=i, qr_fp64=True))
    ops = [api.Operator.kernel(p) for p in plans]

    def batched():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Fs = api.Factorization.factor_batch(plans, ops)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, Fs

    def sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Fs = [api.Factorization.factor(p, o) for p, o in zip(plans, ops)]
        torch.cuda.synchronize()
        return time.perf_counter() - t0, Fs

    batched(), sequential()   # warm-up
    tb = min(batched()[0] for _ in range(reps))
    ts, Fs_seq = min((sequential() for _ in range(reps)), key=lambda r: r[0])
    s0 = api.sync_count()
    _, Fs = batched()
    syncs_b = api.sync_count() - s0
    s0 = api.sync_count()
    sequential()
    syncs_s = api.sync_count() - s0
    errs = [F.error(o, 16, seed=5) for F, o in zip(Fs, ops)]
    bound = max(2 * math.sqrt(p.L + 2) * 1e-5 for p in plans)
    return {"operators": count, "n_total": int(sum(sizes)), "sizes": {str(k): sizes.count(k) for k in sorted(set(sizes))},
            "batched_s": tb, "sequential_s": ts, "speedup": ts / tb,
            "host_syncs_batched": syncs_b, "host_syncs_sequential": syncs_s,
            "max_sketch_error": float(max(errs)), "error_bound": bound,
            "all_within_bound": bool(all(e <= 2 * math.sqrt(p.L + 2) * 1e-5 for e, p in zip(errs, plans)))}


def configs_measure():
    """The other measured configurations, each factorization device-synchronised
    wall time (plan and operator construction excluded), after one warm-up:
    C1 plain FP64 with a dense stored operator (line pair n = m = 1024, A
    materialised on the device by the library's FP64 kernel entries, c128,
    leaf 16, tol 1e-6, p 2, r0 4); C2a exact recovery (random butterfly n =
    16384, leaf 32, rank 8, seed 1, black box = apply of its own factors, FP64,
    tol 1e-12, error must be <= 1e-11); C4 composition (60-degree caps P1, P2,
    P3 on unit spheres at x = -3, 0, 3, n = 65536 each, 8 points per
    wavelength, exp(i k r)/(4 pi r); K1 = K(P2<-P1) and K2 = K(P3<-P2)
    factorized from entries on the fly, then A = K2 K1 recompressed through
    applies only; complex64 sketches, FP64 QR, tol 1e-6, p 4, r0 64, leaf 64)."""
    import torch
    from paper_2002_03400_gb300 import api, inputs

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    res = {}
    # C1
    g = inputs.line_pair(1024)
    p1 = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                  precision="fp64", p=2, r0=4)
    eye = torch.eye(1024, dtype=torch.complex128, device="cuda")
    A = api.Operator.kernel(p1).apply(eye)            # dense A, user order, FP64 entries
    opd = api.Operator.dense(p1, A)
    timed(lambda: api.Factorization.factor(p1, opd))
    t1, F1 = timed(lambda: api.Factorization.factor(p1, opd))
    res["c1_plain_fp64"] = {"factor_s": t1, "sketch_error": F1.error(opd, 16, seed=7),
                            "bound": 2 * math.sqrt(p1.L + 2) * 1e-6, "ranks_max": int(max(F1.ranks(0, 0)))}
    # C2a
    eb = inputs.exact_butterfly(16384, 32, 8, seed=1)
    Fx = api.exact_factorization(api.Plan(n=16384, leaf=32), eb)
    opx = api.Operator.factored(Fx)
    p2 = api.Plan(n=16384, leaf=32, tol=1e-12, precision="fp64")
    timed(lambda: api.Factorization.factor(p2, opx))
    t2, F2 = timed(lambda: api.Factorization.factor(p2, opx))
    res["c2a_exact"] = {"factor_s": t2, "recovery_error": F2.error(opx, 16, seed=7), "required": 1e-11,
                        "ranks": sorted(set(int(r) for r in F2.ranks(0, 0)))}
    # C4
    n = 65536
    P1 = inputs.cap_points(n, (-3.0, 0.0, 0.0), 60.0, axis=(1.0, 0.0, 0.0))
    P2 = inputs.cap_points(n, (0.0, 0.0, 0.0), 60.0, axis=(-1.0, 0.0, 0.0))
    P3 = inputs.cap_points(n, (3.0, 0.0, 0.0), 60.0, axis=(-1.0, 0.0, 0.0))
    k = 2.0 * math.pi / (8.0 * math.sqrt(math.pi / n))
    kw = dict(leaf=64, tol=1e-6, precision="mixed", p=4, r0=64, qr_fp64=True)
    pk1 = api.Plan(P1, P2, kernel="helmholtz3d", wavenumber=k, **kw)
    pk2 = api.Plan(P2, P3, kernel="helmholtz3d", wavenumber=k, **kw)
    ok1, ok2 = api.Operator.kernel(pk1), api.Operator.kernel(pk2)
    tk1, K1 = timed(lambda: api.Factorization.factor(pk1, ok1))
    tk2, K2 = timed(lambda: api.Factorization.factor(pk2, ok2))
    comp = api.Operator.composed(api.Operator.factored(K2), api.Operator.factored(K1))
    pa = api.Plan(P1, P3, **kw)
    ta, FA = timed(lambda: api.Factorization.factor(pa, comp))
    # adjacent hemispheres (Sec. 7.3, Table 2's geometry): touching unit
    # hemispheres, 10 points per wavelength, p 4, r0 64, leaf 64, tol 1e-4
    # (Table 2's tightest), mixed with FP64 QR; factor time, the largest rank
    # per level (the weak-admissibility growth) and the sketch error
    hemi = {}
    for nh in (16384, 65536):
        gh = inputs.hemisphere_pair(nh)
        ph = api.Plan(gh.src, gh.tgt, kernel="helmholtz3d", wavenumber=gh.wavenumber, leaf=64, tol=1e-4, p=4, r0=64,
                      precision="mixed", qr_fp64=True)
        oh = api.Operator.kernel(ph)
        timed(lambda: api.Factorization.factor(ph, oh))
        th, Fh = timed(lambda: api.Factorization.factor(ph, oh))
        hemi[str(nh)] = {"factor_s": th, "L": ph.L,
                         "max_rank_V": [int(Fh.ranks(0, j).max()) for j in range(ph.lm + 1)],
                         "max_rank_U": [int(Fh.ranks(1, j).max()) for j in range(ph.lm, ph.L + 1)],
                         "sketch_error": Fh.error(oh, 16, seed=7, dtype=torch.complex64),
                         "bound": 2 * math.sqrt(ph.L + 2) * 1e-4}
        del Fh, oh, ph
    res["hemispheres_tol1e-4"] = hemi
    res["c4_composition"] = {"n": n, "k1_factor_s": tk1, "k2_factor_s": tk2, "recompress_s": ta,
                             "k1_error": K1.error(ok1, 16, seed=7), "k2_error": K2.error(ok2, 16, seed=7),
                             "recompress_error": FA.error(comp, 16, seed=7),
                             "bound": 2 * math.sqrt(pa.L + 2) * 1e-6,
                             "black_box_columns": list(comp.counts())}
    return res


def max_over_ranks(values, dist=None, device="cpu"):
    """The slowest rank's value of each entry (the step-time rule for N
    replicas: an all-reduce MAX over the process group); the values
    unchanged on one rank (dist None)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, timed on the
    benchmark workload itself (n = 16384; rank 0 only under torchrun, the
    other ranks exit without work).  Warm-up steps are small untimed oracle
    runs (n = 256: imports, BLAS threads, page-in).  Each timed step is one
    full oracle factorization (minutes); the arm runs as many of the
    requested steps as fit in BF_REFERENCE_BUDGET_S seconds (default 300,
    at least one) and prints the number it ran."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # BF_REFERENCE_N: a smaller size for tests of this host path only
    n_ref = int(os.environ.get("BF_REFERENCE_N", str(N)))
    for _ in range(args.warmup):   # untimed
        oracle_factor_seconds(256)
    budget = float(os.environ.get("BF_REFERENCE_BUDGET_S", "300"))
    samples = []
    t_start = time.perf_counter()
    while len(samples) < args.steps:
        samples.append(oracle_factor_seconds(n_ref))
        spent = time.perf_counter() - t_start
        if spent + samples[-1] > budget:
            break
    v = float(np.mean(samples))
    line = {"impl": "reference", "metric": "factor time (s)", "value": v, "unit": "s",
            "n_gpus": args.gpus, "steps": len(samples), "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic", "config": bench_config(n_ref),
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "s", "cores": os.cpu_count(),
                             "sample": f"{len(samples)} full oracle factorization(s) of the benchmark workload "
                                       f"(n = {n_ref}), each timed; {ORACLE_CORES_NOTE}"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 20 steps of ~14 ms: a timed region of ~0.3 s, long enough for the
    # clock sampler (100 ms interval) to see it under load
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--profile-case", choices=["sketch", "apply", "qr", "step", "image"], default=None,
                    help="run only a small case of one kernel family (for ncu captures)")
    ap.add_argument("--engine", default="tensor")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args)

    import torch
    from paper_2002_03400_gb300 import api, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    stream = torch.cuda.current_stream()
    g = inputs.line_pair(N)
    # the measured form: complex64 sketches and peeling, FP64 pivoted QR,
    # truncation and B least squares
    plan_mx = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                       precision="mixed", r0=R0, qr_fp64=True)
    plan_64 = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                       precision="fp64", r0=R0)
    op_mx = api.Operator.kernel(plan_mx)
    op_64 = api.Operator.kernel(plan_64)
    # right-hand sides column-major, the library's layout (no copy per call)
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(N, NRHS, seed=1)).cuda())
    x32 = api.colmajor(x.to(torch.complex64))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(plan, op, xin, ev=None):
        F = api.Factorization.factor(plan, op)
        if ev is not None:
            ev.record(stream)
        y = F.apply(xin)
        err = F.error(op, 16, seed=7, dtype=xin.dtype)
        return F, y, err

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step(plan_mx, op_mx, x32)
    # plain FP64 form, once, for the comparison line
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F64, _, err64 = step(plan_64, op_64, x)
    torch.cuda.synchronize()
    fp64_step_s = time.perf_counter() - t0
    fp64_factor_s = F64.info()["seconds"]

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fac_s, errs = [], []
    # nvidia-smi samples of the timed region: BF_CLOCKS_CSV names the file
    clk = ClockSampler(os.environ.get("BF_CLOCKS_CSV", "/tmp/clocks_bench.csv"))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = api.launch_count()
    syncs0 = api.sync_count()
    with clk:
        for i in range(args.steps):
            flush.fill_(1.0)
            starts[i].record(stream)
            F, y, err = step(plan_mx, op_mx, x32, mids[i])
            ends[i].record(stream)
            fac_s.append(F.info()["seconds"])
            errs.append(err)
        torch.cuda.synchronize()
    gpu_launches = api.launch_count() - launches0
    host_syncs = api.sync_count() - syncs0
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fac_ms = [s.elapsed_time(e) for s, e in zip(starts, mids)]
    ms = float(np.mean(step_ms))
    fms = float(np.mean(fac_ms))
    ms, fms = max_over_ranks([ms, fms], dist, "cuda")

    # apply GB/s (resident factors, complex64 and complex128), after the
    # apply tuner has chosen engine, depth, slice width and stage shapes;
    # each engine beside it.  Device time: a device-side sleep queued ahead
    # of the first event lets the host enqueue every apply before the GPU
    # reaches it, so host launch costs stay outside the timed region.
    def apply_time(F, xin, reps=20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        F.apply(xin)
        torch.cuda.synchronize()
        if hasattr(torch.cuda, "_sleep"):
            torch.cuda._sleep(20_000_000)   # ~10 ms at 2 GHz
        e0.record(stream)
        for _ in range(reps):
            F.apply(xin)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    def apply_gbs(F, xin):
        info = F.info()
        es = 8 if xin.dtype == torch.complex64 else 16
        nr = xin.shape[1]
        byts = info["stored_entries"] * es + nr * (2 * N) * es
        F.tune(nr, xin.dtype)
        t = apply_time(F, xin)               # the tuned choice (engine, depth, slice width, stage shapes)
        other = []
        for eng in ("stages", "fused", "persistent", "grouped"):
            api.set_apply_engine(eng)
            other.append(apply_time(F, xin))
        api.set_apply_engine("auto")
        return byts / t / 1e9, t, byts, tuple(other)

    gbs32, t32, b32, ts32 = apply_gbs(F, x32)
    gbs64, t64, b64, ts64 = apply_gbs(F64, x)
    gbs1, t1, b1, ts1 = apply_gbs(F, x32[:, :1])

    # variants of the same factorization, each timed like the steps (3 runs,
    # the first discarded): the pivoted QR and truncation in float-float
    # (~2^-46, on the FP32 pipe) instead of FP64; and Alg. 2's initial rank
    # guess r0 = 4 (the paper's value) instead of 16, which must give the
    # same factorization (leaf passes append columns of one counter-based
    # stream, so the final leaf sketch is the same)
    def timed_factor(plan, op):
        out = []
        F = None
        for _ in range(3):
            flush.fill_(1.0)
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            F = api.Factorization.factor(plan, op)
            q1.record(stream)
            torch.cuda.synchronize()
            out.append(q0.elapsed_time(q1) / 1e3)
        return float(np.mean(out[1:])), F

    plan_ff = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                       precision="mixed", r0=R0)
    op_ff = api.Operator.kernel(plan_ff)
    t_ff, Fff = timed_factor(plan_ff, op_ff)
    qr_ff = {"factor_s": t_ff, "sketch_error": Fff.error(op_ff, 16, seed=7, dtype=torch.complex64),
             "dtype": "c64 products, float-float (~2^-46) QR and truncation, FP64 B"}
    plan_r4 = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                       precision="mixed", r0=4, qr_fp64=True)
    t_r4, F4 = timed_factor(plan_r4, api.Operator.kernel(plan_r4))
    same_ranks = all(np.array_equal(F4.ranks(0, j), F.ranks(0, j)) for j in range(plan_mx.lm + 1)) and all(
        np.array_equal(F4.ranks(1, j), F.ranks(1, j)) for j in range(plan_mx.lm, plan_mx.L + 1))
    r0_4 = {"factor_s": t_r4, "same_ranks_as_r0_16": bool(same_ranks),
            "same_apply_as_r0_16": bool(same_ranks and torch.equal(F4.apply(x32), F.apply(x32))),
            "black_box_columns": [F4.info()["cols_N"], F4.info()["cols_T"]],
            "black_box_columns_r0_16": [F.info()["cols_N"], F.info()["cols_T"]]}
    del F4, Fff

    # roofline of the dominant kernel of the factorization: the sketch
    # product fed by the complex64 entry image (sketch_img_kernel), one
    # product over all m x n entries at the widest sketch width of the run,
    # timed with CUDA events on the launching stream through an operator
    # whose images are resident; the image formation (entry_images_kernel,
    # one launch for both orientations) is timed when that operator is built
    kw = 22
    Xk = api.colmajor(torch.from_numpy(inputs.random_rhs(N, kw, seed=3)).to(torch.complex64).cuda())
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    torch.cuda.synchronize()
    r0.record(stream)
    op_img = api.Operator.kernel(plan_mx, cached=True)
    r1.record(stream)
    torch.cuda.synchronize()
    t_form = r0.elapsed_time(r1) / 1e3              # both orientations, one pass
    op_img.apply(Xk)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(reps):
        op_img.apply(Xk)
    r1.record(stream)
    torch.cuda.synchronize()
    t_img = r0.elapsed_time(r1) / reps / 1e3
    del op_img
    torch.cuda.synchronize()
    kp = (kw + 7) // 8 * 8
    nr_img = 16 if kp <= 8 else 32 if kp <= 16 else 48 if kp <= 24 else 64
    img_bytes = 8.0 * N * N + 8.0 * N * kw * 2          # the image (8 B per entry) + X + Y
    chunks = (N // 128) * (N // 16)
    img_mma_flops = chunks * 2 * (2.0 * 128 * 16 * 6 * nr_img)   # 2 K steps x 3 MMAs (N = 3, 2, 1 x NR)
    # per 16-column chunk the tensor pipe needs N/2 cycles per MMA (M = 128,
    # K = 16): 2 K steps x (3 + 2 + 1) NR / 2 = 6 NR cycles; one issuing
    # thread sustains at best ~50 cycles per MMA (measured in isolation), so
    # the chunk costs max(6 NR, 6 x 50) cycles at the 2070 MHz clock
    mma_bound_s = chunks * max(6 * nr_img, 6 * 50) / (152 * 2070e6)
    # the on-the-fly product (entries formed in every sketch; still used by
    # products of plain kernel operators and when images do not fit)
    op_mx.apply(Xk)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(reps):
        op_mx.apply(Xk)
    r1.record(stream)
    torch.cuda.synchronize()
    t_sk = r0.elapsed_time(r1) / reps / 1e3
    sk_flops = 8.0 * N * N * kw            # complex multiply-adds x 8 real flops
    engine_ms = {}
    for eng in ("tensor-3xtf32", "tensor-split3", "simt"):
        api.set_sketch_engine(eng)
        op_mx.apply(Xk)
        torch.cuda.synchronize()
        r0.record(stream)
        for _ in range(reps):
            op_mx.apply(Xk)
        r1.record(stream)
        torch.cuda.synchronize()
        engine_ms[eng] = r0.elapsed_time(r1) / reps
    api.set_sketch_engine("tensor")
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
    alu_peak = 152 * 128 * 2070e6 / 1e12        # FP32 lane operations per second (one per clock)
    # the default product uses the exact three-way bf16 split: 6 bf16 products
    # per real product (kind::f16, the measured bf16 peak applies)
    tc_flops = sk_flops * 6
    tc_peak = measured_peaks()[0].get("bf16_tflops", 1900.0)

    # end to end through the C ABI from host buffers
    xh = x32.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan_e = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                      precision="mixed", r0=R0)
    Fe = api.Factorization.factor(plan_e, api.Operator.kernel(plan_e))
    ye = Fe.apply(xh.cuda(non_blocking=True)).cpu()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    serving = serving_measure() if not args.no_serve else None
    batched = batched_measure() if not args.no_batch else None
    configs = configs_measure() if not args.no_configs else None
    peaks, peak_src = measured_peaks()
    clocks = clk.summary()
    line = {
        "metric": "factor time (s)",
        "value": fms / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64+f64",
        "dtype_detail": "complex64 sketch products and peeling (tensor cores, exact three-way bf16 split, "
                        "FP32 accumulation), FP64 pivoted QR, truncation and B least squares",
        "data": "synthetic",
        "config": bench_config(),
        "factor_s_mixed": float(np.mean(fac_s)),
        "factor_s_fp64": fp64_factor_s,
        "mixed_with_float_float_qr": qr_ff,
        "r0_4": r0_4,
        "sketch_error_mixed": float(np.mean(errs)),
        "sketch_error_fp64": err64,
        "apply_gbs_c64": gbs32,
        "apply_gbs_c128": gbs64,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(xh.numel() * 8 + 2 * N * 2 * 8),
                "d2h_bytes_per_step": int(ye.numel() * 8)},
        "clocks": clocks,
        "gpu_launches": gpu_launches,
        "gpu_launches_per_step": gpu_launches / max(1, args.steps),
        "host_syncs_per_step": host_syncs / max(1, args.steps),
        "peaks_source": peak_src,
        "serving": serving,
        "batched": batched,
        "configs": configs,
        "roofline": {"kernel": "sketch_img_kernel (tcgen05, complex64 entry image streamed, exact three-way "
                               "bf16 split, B parts stacked along N)", "bound": "hbm",
                     "achieved": img_bytes / t_img / 1e9, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                     "frac": img_bytes / t_img / 1e9 / peaks.get("hbm_gbs", 6800.0),
                     "traffic": IMG_TRAFFIC_N8192 * (N / 8192) ** 2 if img_traffic_valid() else None,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at "
                                        "n = 8192, scaled by the entry count to n = 16384"
                                        if img_traffic_valid() else
                                        "null: the kernel source changed since the last ncu capture"),
                     "peak_source": peak_src + " (burst copy)",
                     "work": f"8 B per entry of the m=n={N} image + the {kw}-column X and Y, once each; "
                             "the timed product is 3 launches (B operand, image sketch, split-K reduce)",
                     "launch_ms": t_img * 1e3,
                     "tensor_pipe": {"achieved_tflops": img_mma_flops / t_img / 1e12, "peak_tflops": tc_peak,
                                     "frac": img_mma_flops / t_img / 1e12 / tc_peak,
                                     "peak_source": "measured bf16 (burst)",
                                     "mma_bound_ms": mma_bound_s * 1e3,
                                     "frac_of_mma_bound": mma_bound_s / t_img},
                     "entry_images_kernel": {"bound": "alu", "ms_both_orientations": t_form * 1e3,
                                             "achieved": ALU_OPS_PER_ENTRY * N * N / t_form / 1e12,
                                             "peak": alu_peak, "unit": "Tops/s",
                                             "frac": ALU_OPS_PER_ENTRY * N * N / t_form / 1e12 / alu_peak,
                                             "hbm_gbs": 16.0 * N * N / t_form / 1e9,
                                             "work": f"{ALU_OPS_PER_ENTRY} FP32 ops per entry (the float-float "
                                                     "formula, once for both images) + 16 B written"},
                     "on_the_fly": {"kernel": "sketch_tc_kernel (entries formed in the product)", "bound": "alu",
                                    "launch_ms": t_sk * 1e3, "engine_ms": engine_ms,
                                    "achieved": ALU_OPS_PER_ENTRY * N * N / t_sk / 1e12, "peak": alu_peak,
                                    "unit": "Tops/s", "frac": ALU_OPS_PER_ENTRY * N * N / t_sk / 1e12 / alu_peak,
                                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz",
                                    "tensor_frac": tc_flops / t_sk / 1e12 / tc_peak},
                     "apply": {"kernel": "the tuned apply engine (the fastest measured of: grouped runs of stages "
                                         "per launch, stage launches, the fused two-launch engine, the "
                                         "persistent cooperative launch)",
                               "bound": "alu (complex64, 64 RHS: 4 FP32 FMA per factor entry and column; "
                                        "the HBM fraction is reported beside it)",
                               "achieved_gbs_c64": gbs32, "peak_gbs": peaks.get("hbm_gbs"),
                               "frac_c64": gbs32 / peaks.get("hbm_gbs", 6800.0),
                               # 4 real FMAs per stored factor entry and column (one complex
                               # multiply-add); FP32 lanes: 152 SMs x 128 x 2070 MHz; FP64: 2
                               # FMAs per clock per SM (the nominal 1.25 TFLOP/s)
                               "fma_frac_c64": 4.0 * F.info()["stored_entries"] * NRHS / t32
                                               / (152 * 128 * 2070e6),
                               "fma_frac_c128": 4.0 * F64.info()["stored_entries"] * NRHS / t64
                                                / (152 * 2 * 2070e6),
                               "achieved_gbs_c128": gbs64, "frac_c128": gbs64 / peaks.get("hbm_gbs", 6800.0),
                               "bytes_per_apply_c64": b32, "bytes_per_apply_c128": b64,
                               "ms_c64": t32 * 1e3, "ms_c128": t64 * 1e3, "ms_c64_1rhs": t1 * 1e3,
                               "gbs_c64_1rhs": gbs1,
                               "stage_engine_ms": {"c64": ts32[0] * 1e3, "c128": ts64[0] * 1e3,
                                                   "c64_1rhs": ts1[0] * 1e3},
                               "fused_engine_ms": {"c64": ts32[1] * 1e3, "c128": ts64[1] * 1e3,
                                                   "c64_1rhs": ts1[1] * 1e3},
                               "persistent_engine_ms": {"c64": ts32[2] * 1e3, "c128": ts64[2] * 1e3,
                                                        "c64_1rhs": ts1[2] * 1e3},
                               "grouped_engine_ms": {"c64": ts32[3] * 1e3, "c128": ts64[3] * 1e3,
                                                     "c64_1rhs": ts1[3] * 1e3},
                               "work": f"factor entries + {NRHS} input and {NRHS} output columns, once each"}},
    }
    if rank == 0 and not args.no_cpu:
        # the oracle as it stands, once, on the benchmark workload itself
        # (after the GPU work: nothing else runs on the host meanwhile)
        t_or = oracle_factor_seconds(N)
        line["cpu_baseline"] = {"value": t_or, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"one full oracle factorization of the benchmark workload (n = {N}), "
                                          f"timed; {ORACLE_CORES_NOTE}"}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
