"""Host logic of the serving loop (no GPU): request traces, job construction,
latency statistics, memory estimates."""
import numpy as np

from paper_2002_03400_gb300 import inputs, serve


def test_trace_is_poisson_and_seeded():
    tr = inputs.serving_trace(duration_s=200.0, rate_hz=50.0, seed=1, resident=4)
    assert tr == inputs.serving_trace(duration_s=200.0, rate_hz=50.0, seed=1, resident=4)
    gaps = np.diff([r.t for r in tr])
    assert abs(len(tr) / 200.0 - 50.0) < 5 * np.sqrt(50 / 200.0) * 3
    assert abs(gaps.mean() - 1 / 50) < 0.003 and abs(gaps.std() - 1 / 50) < 0.004   # exponential
    frac = np.mean([r.kind == "apply" for r in tr])
    assert abs(frac - 0.8) < 0.03
    ap = [r for r in tr if r.kind == "apply"]
    assert min(r.nrhs for r in ap) >= 1 and max(r.nrhs for r in ap) <= 64
    assert {r.dtype for r in ap} == {"c64", "c128"}
    assert {r.target for r in tr if r.kind == "factor"} <= {4096, 16384, 65536}


def test_jobs_and_latency_stats():
    tr = inputs.serving_trace(duration_s=2.0, rate_hz=30.0, seed=2, resident=2)
    jobs = serve.make_jobs(tr, ["a", "b"], {"a": 100, "b": 200}, seed=0)
    for j, r in zip(jobs, tr):
        assert j.kind == r.kind and j.t_arrive == r.t
        if j.kind == "apply":
            assert j.x.shape == ({"a": 100, "b": 200}[j.target], r.nrhs)
            assert j.x.dtype == (np.complex64 if r.dtype == "c64" else np.complex128)
    for i, j in enumerate(jobs):
        j.t_done = j.t_arrive + 0.001 * (i + 1)
    st = serve.latency_stats(jobs)
    lat = np.array([0.001 * (i + 1) for i in range(len(jobs))])
    assert abs(st["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9


def test_memory_estimate_grows_like_n_log_n():
    a, b = serve.estimate_bytes(4096), serve.estimate_bytes(65536)
    assert 16 * 1.0 < b / a < 16 * 2.0
