"""The fused apply (two launches: one CTA per subtree and column slice on
each side of the centre level, eq. hybrid_butterfly_mat split as in the
paper's hybrid layout, Sec. 6.2) against the stage engine and the oracle.

Every output of the fused kernels is the same sequential FMA chain as in
the stage kernels, so the two engines must agree bit for bit: for y = F x,
F^T x and F^H x, complex64 and complex128, column counts that span one and
several column slices with a ragged last slice, leading dimensions larger
than the row count, permuted and ragged trees, and hybrid levels 0 and
L - 1 (one side of the split is then a single subtree).  The apply tuner
may switch engines and slice widths per right-hand-side class, never the
result."""
import numpy as np
import pytest
import torch

from oracle import butterfly as ob
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _engine():
    yield
    api.set_apply_engine("auto")


def _cases():
    eb = inputs.exact_butterfly(2048, 32, 8, seed=1)
    yield "exact", api.exact_factorization(api.Plan(n=2048, leaf=32), eb), eb
    g = inputs.cap_pair(777, m=700)
    p = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, precision="mixed")
    yield "cap-ragged", api.Factorization.factor(p, api.Operator.kernel(p)), None
    g = inputs.arc_pair(1000, seed=3, m=900)
    p = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=16, tol=1e-6, precision="mixed")
    yield "arc-ragged", api.Factorization.factor(p, api.Operator.kernel(p)), None
    g = inputs.line_pair(1024)
    for hl in (0, 5):
        p = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                     precision="mixed", hybrid_level=hl)
        yield f"line-hybrid{hl}", api.Factorization.factor(p, api.Operator.kernel(p)), None


def _apply(F, x, op, engine):
    api.set_apply_engine(engine)
    y = F.apply(x, op)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("case", ["exact", "cap-ragged", "arc-ragged", "line-hybrid0", "line-hybrid5"])
def test_fused_equals_stages_bit_for_bit(case):
    name, F, eb = next(c for c in _cases() if c[0] == case)
    n, m = F.plan.n, F.plan.m
    for dt in (torch.complex128, torch.complex64):
        for nrhs in (1, 3, 16, 37, 64):
            for op in ("N", "T", "C"):
                rows = n if op == "N" else m
                big = torch.from_numpy(inputs.random_rhs(rows + 5, nrhs, seed=nrhs)).to(dt).cuda()
                x = api.colmajor(big)[:rows]                       # ld = rows + 5
                yf = _apply(F, x, op, "fused")
                ys = _apply(F, x, op, "stages")
                assert torch.equal(yf, ys), (case, dt, nrhs, op)
                if eb is not None and dt == torch.complex128:
                    yo = ob.apply(ob.from_blocks(eb), x.cpu().numpy(), op)
                    assert np.linalg.norm(yf.cpu().numpy() - yo) <= 1e-13 * np.linalg.norm(yo)


def test_tuning_keeps_results():
    g = inputs.line_pair(4096)
    p = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6, precision="mixed")
    F = api.Factorization.factor(p, api.Operator.kernel(p))
    for dt in (torch.complex64, torch.complex128):
        for nrhs in (1, 64):
            x = api.colmajor(torch.from_numpy(inputs.random_rhs(4096, nrhs, seed=2)).to(dt).cuda())
            y0 = _apply(F, x, "N", "fused")
            api.set_apply_engine("auto")
            ms = F.tune(nrhs, dt)
            assert ms > 0
            assert torch.equal(_apply(F, x, "N", "auto"), y0)
            assert torch.equal(_apply(F, x, "N", "fused"), y0)
            assert torch.equal(_apply(F, x, "N", "stages"), y0)
