"""Every stage-kernel shape of the apply computes the same sums in the same
order (terms in order, k ascending, one FMA chain per output), so forcing
any one of them for every stage leaves F x, F^T x and F^H x unchanged bit
for bit (eq. hybrid_butterfly_mat).  Column counts cover one column, partial
and whole 64-column slices and more than one slice; the trees are ragged and
permuted (arc pair, leaf 24), so blocks of every rank and odd row offsets
occur."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _reset_variant():
    yield
    api.set_stage_variant(-1)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_every_stage_variant_bit_identical(dtype):
    n = 1500
    g = inputs.arc_pair(n, seed=11)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6,
                    precision="mixed" if dtype == torch.complex64 else "fp64")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    for nrhs in (1, 3, 37, 64, 130):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(n, nrhs, seed=nrhs)).to(dtype).cuda())
        api.set_stage_variant(-1)
        ref = {op: F.apply(x, op=op).cpu().numpy() for op in ("N", "T", "C")}
        for v in range(api.STAGE_VARIANTS):
            api.set_stage_variant(v)
            for op in ("N", "T", "C"):
                got = F.apply(x, op=op).cpu().numpy()
                assert np.array_equal(got, ref[op]), (v, nrhs, op)


def test_stage_variant_rejects_out_of_range():
    with pytest.raises(api.BFError):
        api.set_stage_variant(api.STAGE_VARIANTS)
    with pytest.raises(api.BFError):
        api.set_stage_variant(-2)
