"""Serving: continuous batching over resident factorizations.

Every request served in the mix (coalesced applies, factorizations running
on worker streams at the same time) must return what it returns alone."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs, serve

pytestmark = pytest.mark.gpu


def _resident():
    out = {}
    for name, (n, geo, prec) in {"a": (1024, "arc", "mixed"), "b": (2048, "arc", "fp64"),
                                 "c": (1500, "cap", "mixed")}.items():
        spec = serve.factor_spec(n, geo, seed=len(out), precision=prec)
        out[name] = (serve.build_factor(spec), n)
    return out


def test_each_result_is_the_same_alone_and_in_the_mix():
    res = _resident()
    trace = inputs.serving_trace(duration_s=0.5, rate_hz=200, seed=4, resident=3, factor_sizes=(1024, 2048),
                                 apply_fraction=0.9)
    names = list(res)
    jobs = serve.make_jobs(trace, names, {k: v[1] for k, v in res.items()}, seed=1)
    assert sum(j.kind == "factor" for j in jobs) >= 1 and len(jobs) > 40
    srv = serve.Server(mem_cap=8e9, factor_workers=2)
    for k, (F, _) in res.items():
        srv.add_resident(k, F)
    done = srv.run(jobs, realtime=True)
    srv.close()
    assert len(done) == len(jobs) and all(not j.error for j in done)
    coalesced = 0
    for j in done:
        if j.kind == "apply":
            F = res[j.target][0]
            dt = torch.complex64 if j.dtype == "c64" else torch.complex128
            alone = F.apply(torch.from_numpy(j.x).to(dt).cuda()).cpu().numpy()
            assert np.array_equal(alone, j.result), j.rid     # bit for bit
        else:
            Fa = serve.build_factor(j.spec)
            x = torch.from_numpy(inputs.random_rhs(j.spec["n"], 3, seed=7)).cuda()
            ya, ym = Fa.apply(x).cpu().numpy(), j.result.apply(x).cpu().numpy()
            assert np.array_equal(ya, ym), j.rid
    stats = serve.latency_stats(done)
    assert stats["p50_ms"] is not None and stats["p99_ms"] >= stats["p50_ms"]


def test_admission_waits_for_memory_and_evicts_idle_factors():
    spec = serve.factor_spec(1024, "arc", seed=3)
    est = serve.estimate_bytes(1024)
    srv = serve.Server(mem_cap=1.5 * est, factor_workers=2)
    jobs = [serve.Job(0, "factor", 0.0, "f0", spec=spec), serve.Job(1, "factor", 0.0, "f1", spec=spec),
            serve.Job(2, "factor", 0.0, "f2", spec=spec)]
    done = srv.run(jobs, realtime=False)
    srv.close()
    assert all(j.result is not None for j in done)
    # the cap admits one factorization at a time; the others waited
    assert srv.peak_inflight == est
    assert srv.used_bytes() <= srv.mem_cap
