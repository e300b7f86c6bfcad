"""Graph-captured apply (bf_applier): the same stage chain as bf_apply,
captured once into a CUDA graph, so every result equals bf_apply's bit for
bit -- for every op, both dtypes, ragged trees with non-identity
permutations, and runs issued from two streams."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("op", ["N", "T", "C"])
def test_applier_equals_apply(dtype, op):
    g = inputs.cap_pair(1500, m=1300)          # ragged trees, permuted points
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, p=4,
                    precision="mixed" if dtype == torch.complex64 else "fp64")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    rows_in = 1500 if op == "N" else 1300
    for nrhs in (1, 7, 64):
        F.tune(nrhs, dtype, op=op)
        A = F.applier(nrhs, dtype, op)
        for seed in (1, 2):
            x = api.colmajor(torch.from_numpy(inputs.random_rhs(rows_in, nrhs, seed=seed)).to(dtype).cuda())
            want = F.apply(x, op=op).cpu().numpy()
            got = A.run(x).cpu().numpy()
            assert np.array_equal(got, want)
        A.free()


def test_applier_runs_from_two_streams_and_rejects_bad_input():
    g = inputs.arc_pair(2048, seed=4)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, precision="mixed")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    A = F.applier(16)
    xs = [api.colmajor(torch.from_numpy(inputs.random_rhs(2048, 16, seed=s)).to(torch.complex64).cuda())
          for s in range(6)]
    want = [F.apply(x).cpu().numpy() for x in xs]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    ys = []
    for i, x in enumerate(xs):
        st = s1 if i % 2 == 0 else s2
        with torch.cuda.stream(st):
            ys.append(A.run(x, stream=st))
    torch.cuda.synchronize()
    for y, w in zip(ys, want):
        assert np.array_equal(y.cpu().numpy(), w)
    with pytest.raises(ValueError):
        A.run(xs[0][:, :8])
    bad = api.empty_cm(100, 16, torch.complex64, "cuda")
    with pytest.raises(api.BFError):   # ld below the row count
        api.check(api.lib().bf_applier_run(A._h, bad.data_ptr(), 100, bad.data_ptr(), 100, None))
