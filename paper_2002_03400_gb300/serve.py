"""Continuous-batching request loop over resident butterfly factorizations.

Requests are applies (y = F x with 1..64 right-hand sides, complex64 or
complex128) against factorizations kept resident on the device, and new
factorizations (bf_factor of a kernel operator on some geometry).  The loop

* admits a request only when a slot is free and its device memory fits
  under the cap (estimated before, measured after a factorization; idle
  resident factorizations are evicted least-recently-used when needed);
* coalesces the queued applies of one factorization and dtype into one
  multi-right-hand-side bf_apply on the apply stream, so requests that arrive
  while earlier work is on the GPU join the next launch;
* runs factorizations on worker threads, each with its own CUDA stream (the
  library releases the interpreter lock), overlapping them with the applies,
  which run on a high-priority stream so that they do not queue behind a
  factorization's long launches;
* completes requests through CUDA events and reports per-request latency
  (arrival to result on the host) with p50/p99 and throughput.

Every result equals what the same request returns when served alone: the
apply's block products are computed column by column, and a factorization's
arithmetic does not depend on what else runs on the device.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
import time
from collections import OrderedDict, defaultdict
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, inputs


@dataclass
class Job:
    rid: int
    kind: str                    # "apply" | "factor"
    t_arrive: float              # seconds on the server clock
    target: str = ""             # resident name (apply) / new name (factor)
    x: np.ndarray | None = None  # host right-hand sides (apply)
    dtype: str = "c128"
    spec: dict = field(default_factory=dict)   # factor: geometry / plan parameters
    t_done: float = -1.0
    result: object = None
    error: str = ""


class _Rows:
    """Pinned result rows of one launch (and its pinned inputs, kept alive
    until the launch completes)."""

    def __init__(self, yh: torch.Tensor, xh: torch.Tensor):
        self.yh, self.xh = yh, xh

    def cols(self, c0: int, nc: int) -> np.ndarray:
        return self.yh[c0:c0 + nc].numpy().T.copy()


def factor_spec(n: int, geometry: str, seed: int, precision: str = "mixed", tol: float = 1e-6,
                qr_fp64: bool = True) -> dict:
    """Plan parameters of a factor request: arcs (leaf 32) or caps (leaf 64);
    mixed precision with the pivoted QR in FP64 by default."""
    return {"n": n, "geometry": geometry, "seed": seed, "precision": precision, "tol": tol, "qr_fp64": qr_fp64}


def build_factor(spec: dict, stream=None) -> api.Factorization:
    n = spec["n"]
    if spec["geometry"] == "arc":
        g = inputs.arc_pair(n, seed=spec["seed"])
        leaf = 32
    else:
        g = inputs.cap_pair(n)
        leaf = 64
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=leaf, tol=spec["tol"],
                    precision=spec["precision"], p=2 if spec["geometry"] == "arc" else 4,
                    r0=4 if spec["geometry"] == "arc" else 64, seed=spec["seed"],
                    qr_fp64=bool(spec.get("qr_fp64", False)) and spec["precision"] == "mixed")
    return api.Factorization.factor(plan, api.Operator.kernel(plan), stream=stream)


def estimate_bytes(n: int) -> int:
    """Device bytes of a factorization of size n before it exists (factors in
    complex128 and complex64 plus sketch workspace), generous."""
    L = max(1, int(np.ceil(np.log2(max(n, 2) / 32))))
    return int(24 * n * 64 * (2 * L + 3) + 64 * n * 64 * 16)


def fact_bytes(F: api.Factorization) -> int:
    return int(F.info()["stored_entries"] * 24)


class Server:
    def __init__(self, mem_cap: float = 150e9, factor_workers: int = 2, max_cols: int = 512,
                 coalesce: bool = True, apply_slots: int = 4):
        self.mem_cap = mem_cap
        self.max_cols = max_cols
        self.coalesce = coalesce
        self.apply_slots = apply_slots
        self.resident: OrderedDict[str, api.Factorization] = OrderedDict()
        self.res_bytes: dict[str, int] = {}
        self.inflight_bytes = 0
        self.peak_inflight = 0
        # applies on a high-priority stream: while a factorization's kernels
        # hold the SMs, the block scheduler places an apply's CTAs first as
        # SMs free up (priorities order scheduling only, never results)
        self.apply_stream = torch.cuda.Stream(priority=-16)
        self.pool = cf.ThreadPoolExecutor(max_workers=factor_workers)
        self.worker_streams = {}
        self.lock = threading.Lock()
        self.t0 = time.perf_counter()

    # -- clock, memory ---------------------------------------------------
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def used_bytes(self) -> int:
        return sum(self.res_bytes.values()) + self.inflight_bytes

    def add_resident(self, name: str, F: api.Factorization):
        with self.lock:
            self.resident[name] = F
            self.res_bytes[name] = fact_bytes(F)

    def _evict_for(self, need: int, busy: set) -> bool:
        while self.used_bytes() + need > self.mem_cap:
            victim = next((k for k in self.resident if k not in busy), None)
            if victim is None:
                return False
            self.resident.pop(victim).free()
            self.res_bytes.pop(victim)
        return True

    # -- factor requests (worker threads) ----------------------------------
    def _factor(self, job: Job, est: int):
        tid = threading.get_ident()
        s = self.worker_streams.setdefault(tid, torch.cuda.Stream())
        try:
            job.result = build_factor(job.spec, stream=s)   # returns after its stream drained
        except Exception as e:          # reported on the job, the loop goes on
            job.error = str(e)
        with self.lock:
            self.inflight_bytes -= est
            if job.result is not None:
                self.resident[job.target] = job.result
                self.res_bytes[job.target] = fact_bytes(job.result)
        job.t_done = self.now()
        return job

    # -- the loop ----------------------------------------------------------
    def run(self, jobs: list[Job], realtime: bool = True) -> list[Job]:
        """Serves `jobs` (sorted by arrival).  With realtime, a job becomes
        visible at its arrival time on the server clock; otherwise all at once."""
        self.t0 = time.perf_counter()
        pending = list(jobs)
        queue: list[Job] = []
        futures = []
        inflight = []                    # (event, [(job, col0, ncols)], y_host, dtype)
        done: list[Job] = []
        i = 0
        while i < len(pending) or queue or futures or inflight:
            time.sleep(0.00005)
            t = self.now()
            while i < len(pending) and (not realtime or pending[i].t_arrive <= t):
                queue.append(pending[i])
                i += 1
            # completions of applies
            still = []
            for ev, parts, yh, dt in inflight:
                if ev.query():
                    tnow = self.now()
                    for job, c0, nc in parts:
                        job.result = yh.cols(c0, nc)
                        job.t_done = tnow
                        done.append(job)
                else:
                    still.append((ev, parts, yh, dt))
            inflight = still
            # completions of factorizations
            fut_still = []
            for f in futures:
                if f.done():
                    done.append(f.result())
                else:
                    fut_still.append(f)
            futures = fut_still
            # admit factor requests by memory
            busy = {j.target for j in queue if j.kind == "apply"}
            rest = []
            for job in queue:
                if job.kind != "factor":
                    rest.append(job)
                    continue
                est = estimate_bytes(job.spec["n"])
                with self.lock:
                    ok = self._evict_for(est, busy)
                    if ok:
                        self.inflight_bytes += est
                        self.peak_inflight = max(self.peak_inflight, self.inflight_bytes)
                if ok:
                    futures.append(self.pool.submit(self._factor, job, est))
                else:
                    rest.append(job)
            queue = rest
            # coalesce applies per (factorization, dtype) into launches
            if len(inflight) < self.apply_slots:
                groups = defaultdict(list)
                rest = []
                for job in queue:
                    if job.kind == "apply" and job.target in self.resident:
                        groups[(job.target, job.dtype)].append(job)
                    else:
                        rest.append(job)
                queue = rest
                for (name, dt), js in groups.items():
                    while js:
                        take, cols = [], 0
                        while js and (not take or (self.coalesce and cols + js[0].x.shape[1] <= self.max_cols)):
                            take.append(js.pop(0))
                            cols += take[-1].x.shape[1]
                        inflight.append(self._launch_apply(name, dt, take))
                        if not self.coalesce:
                            break
                    queue.extend(js)
        return sorted(done, key=lambda j: j.rid)

    def _launch_apply(self, name: str, dt: str, jobs: list[Job]):
        F = self.resident[name]
        self.resident.move_to_end(name)
        tdt = torch.complex64 if dt == "c64" else torch.complex128
        # right-hand sides as rows of a pinned buffer (its transpose is the
        # column-major n x ncols matrix the library takes), each request's
        # columns copied straight into it (one host copy; the pinned blocks
        # come from torch's caching host allocator)
        ncols = sum(j.x.shape[1] for j in jobs)
        xh = torch.empty((ncols, F.n), dtype=tdt, pin_memory=True)
        r0 = 0
        for j in jobs:
            xh[r0:r0 + j.x.shape[1]].numpy()[...] = j.x.T
            r0 += j.x.shape[1]
        yh = torch.empty((ncols, F.m), dtype=tdt, pin_memory=True)
        with torch.cuda.stream(self.apply_stream):
            xd = xh.to("cuda", non_blocking=True)
            yd = F.apply(xd.t(), stream=self.apply_stream)
            yh.copy_(yd.t(), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.apply_stream)
        parts, c0 = [], 0
        for j in jobs:
            parts.append((j, c0, j.x.shape[1]))
            c0 += j.x.shape[1]
        return ev, parts, _Rows(yh, xh), dt

    def close(self):
        self.pool.shutdown(wait=True)


def latency_stats(jobs: list[Job]) -> dict:
    lat = np.array([j.t_done - j.t_arrive for j in jobs if j.t_done >= 0])
    ap = [j for j in jobs if j.kind == "apply" and j.t_done >= 0]
    span = max((j.t_done for j in jobs), default=0.0) - min((j.t_arrive for j in jobs), default=0.0)
    return {"requests": len(jobs), "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "applies_per_s": len(ap) / span if span > 0 else None,
            "apply_rhs_per_s": sum(j.x.shape[1] for j in ap) / span if span > 0 else None,
            "errors": sum(1 for j in jobs if j.error)}


def throughput_stats(jobs: list[Job], makespan: float) -> dict:
    """Capacity figures of a run whose requests were all queued at once:
    requests, applies, right-hand sides and factorizations per second over
    the makespan."""
    ok = [j for j in jobs if j.t_done >= 0 and not j.error]
    ap = [j for j in ok if j.kind == "apply"]
    fa = [j for j in ok if j.kind == "factor"]
    return {"makespan_s": makespan, "requests_per_s": len(ok) / makespan, "applies_per_s": len(ap) / makespan,
            "apply_rhs_per_s": sum(j.x.shape[1] for j in ap) / makespan, "factors_per_s": len(fa) / makespan,
            "factor_sizes": sorted({int(j.spec["n"]) for j in fa}), "errors": sum(1 for j in jobs if j.error)}


def make_jobs(trace, names: list[str], n_resident_of: dict, seed: int = 0) -> list[Job]:
    """Jobs for an inputs.serving_trace: applies draw right-hand sides sized
    for their target; factor requests get fresh names."""
    jobs = []
    for rid, rq in enumerate(trace):
        if rq.kind == "apply":
            name = names[rq.target % len(names)]
            x = inputs.random_rhs(n_resident_of[name], rq.nrhs, seed=seed * 100003 + rid,
                                  dtype=np.complex64 if rq.dtype == "c64" else np.complex128)
            jobs.append(Job(rid, "apply", rq.t, name, x, rq.dtype))
        else:
            jobs.append(Job(rid, "factor", rq.t, f"new{rid}",
                            spec=factor_spec(rq.target, rq.geometry, seed=rid)))
    return jobs
