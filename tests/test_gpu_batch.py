"""Batched, level-synchronous factorization (bf_factor_batch) across
operators of uneven size, depth and rank.

Batching changes only how blocks are grouped into launches, not the
arithmetic of any block, so every batched factorization must equal the one
bf_factor computes for the same plan and operator (same ranks, bit-identical
apply), and must stay within the oracle tolerances."""
import math

import numpy as np
import pytest
import torch

from oracle import butterfly as ob
from oracle import operators as oo
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def T(x, dtype=torch.complex128):
    return torch.from_numpy(np.asarray(x)).to(dtype).cuda()


def H(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def _plans(precision, tol):
    out = []
    for i, n in enumerate([512, 1024, 2048, 1024, 768]):
        g = inputs.arc_pair(n, seed=10 + i)
        out.append((g, api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=tol,
                                precision=precision, seed=i)))
    g = inputs.cap_pair(600, m=500)
    out.append((g, api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=tol,
                            precision=precision, seed=9)))
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("mixed", 1e-5)])
def test_batch_equals_individual(precision, tol):
    items = _plans(precision, tol)
    plans = [p for _, p in items]
    assert len({p.L for p in plans}) >= 3          # uneven depths in one batch
    ops = [api.Operator.kernel(p) for p in plans]
    Fb = api.Factorization.factor_batch(plans, ops)
    for (g, p), op, F in zip(items, ops, Fb):
        Fi = api.Factorization.factor(p, api.Operator.kernel(p))
        for j in range(p.lm + 1):
            assert np.array_equal(F.ranks(0, j), Fi.ranks(0, j))
        for j in range(p.lm, p.L + 1):
            assert np.array_equal(F.ranks(1, j), Fi.ranks(1, j))
        x = inputs.random_rhs(p.n, 3, seed=p.n)
        yb, yi = H(F.apply(T(x))), H(Fi.apply(T(x)))
        # every launch takes the same arithmetic per job and block whatever
        # else it carries (split-K and split depth are decided per job)
        assert np.array_equal(yb, yi)
        assert F.error(op, 16, seed=2) <= 2 * math.sqrt(p.L + 2) * tol


def test_batch_of_both_split_depths_equals_individual():
    """Mixed-precision plans with tolerances on both sides of the split-depth
    switch (3xTF32 at 1e-5, the three-way split at 1e-6) and uneven sketch
    widths in one batch: each result is bit-identical to bf_factor's."""
    plans = []
    for i, (n, tol) in enumerate([(1024, 1e-5), (1024, 1e-6), (2048, 1e-5), (768, 1e-6)]):
        g = inputs.arc_pair(n, seed=30 + i)
        plans.append(api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=tol,
                              precision="mixed", seed=i))
    Fb = api.Factorization.factor_batch(plans, [api.Operator.kernel(p) for p in plans])
    for p, F in zip(plans, Fb):
        Fi = api.Factorization.factor(p, api.Operator.kernel(p))
        x = T(inputs.random_rhs(p.n, 2, seed=1))
        assert np.array_equal(H(F.apply(x)), H(Fi.apply(x)))


def test_batch_mixed_operator_kinds_and_oracle():
    """Kernel, dense and black-box (factored) operators in one batch; the
    dense member is checked against the oracle."""
    eps = 1e-6
    g1 = inputs.line_pair(1024)
    A1 = oo.kernel_entries(oo.HELMHOLTZ_2D, g1.wavenumber, g1.tgt, g1.src)
    p1 = api.Plan(g1.src, g1.tgt, kernel="helmholtz2d", wavenumber=g1.wavenumber, leaf=16, tol=eps)
    g2 = inputs.arc_pair(700, seed=3)
    p2 = api.Plan(g2.src, g2.tgt, kernel="helmholtz2d", wavenumber=g2.wavenumber, leaf=16, tol=eps)
    eb = inputs.exact_butterfly(1024, 16, 5, seed=6)
    Fx = api.exact_factorization(api.Plan(n=1024, leaf=16), eb)
    p3 = api.Plan(n=1024, leaf=16, tol=1e-12)
    ops = [api.Operator.dense(p1, T(A1)), api.Operator.kernel(p2), api.Operator.factored(Fx)]
    F1, F2, F3 = api.Factorization.factor_batch([p1, p2, p3], ops)
    Fo = ob.factor(oo.DenseOp(A1), g1.src, g1.tgt, p1.L, eps, 2, 4, seed=0)
    Om = ob.error_probe(1024, 11, 16)
    gap = np.linalg.norm(H(F1.apply(T(Om))) - ob.apply(Fo, Om)) / np.linalg.norm(A1 @ Om)
    assert gap <= 1e-6
    assert F3.error(ops[2], 16, seed=4) <= 1e-11
    for j in range(p3.lm + 1):
        assert np.all(F3.ranks(0, j) == 5)


def test_batch_rejects_mixed_precision_and_bad_entries():
    g = inputs.arc_pair(512, seed=1)
    a = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=32, precision="fp64")
    b = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=32, precision="mixed")
    with pytest.raises(api.BFError) as e:
        api.Factorization.factor_batch([a, b])
    assert e.value.code == -1
