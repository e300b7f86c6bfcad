"""Apply autotuner (bf_apply_tune): the stage-kernel shapes it chooses among
compute identical sums, so tuning never changes a result, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_tuning_keeps_every_result(dtype):
    g = inputs.arc_pair(2048, seed=5)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=1e-6,
                    precision="mixed" if dtype == torch.complex64 else "fp64")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    for nrhs in (1, 3, 16, 40, 64, 80):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(2048, nrhs, seed=nrhs)).to(dtype).cuda())
        before = F.apply(x).cpu().numpy()
        before_c = F.apply(x, op="C").cpu().numpy()
        ms = F.tune(nrhs, dtype)
        ms_c = F.tune(nrhs, dtype, op="C")
        assert ms > 0 and ms_c > 0
        assert np.array_equal(F.apply(x).cpu().numpy(), before)
        assert np.array_equal(F.apply(x, op="C").cpu().numpy(), before_c)


def test_tune_rejects_bad_arguments():
    g = inputs.arc_pair(512, seed=1)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32)
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    with pytest.raises(api.BFError):
        F.tune(0)
    with pytest.raises(api.BFError):   # op outside N / T / C
        api.check(api.lib().bf_apply_tune(F._h, 7, 4, 0, None, None))
