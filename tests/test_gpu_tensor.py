"""Tensor-core (tcgen05, 3xTF32) sketch products against the SIMT FP32 path
and FP64, and a mixed-precision factorization on them against the oracle.

Accuracy model: 3xTF32 drops the lo*lo term and rounds each half to 11
significant bits, so a product carries ~2^-21 relative error; the TwoSum
drain of the accumulator after every 32-point chunk keeps the long sums at
that level.  Tolerance on a sketch product: 2e-6 relative to its norm."""
import math

import numpy as np
import pytest
import torch

from oracle import butterfly as ob
from oracle import operators as oo
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def T(x, dtype=torch.complex64):
    return api.colmajor(torch.from_numpy(np.asarray(x)).to(dtype).cuda())


def H(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(autouse=True)
def _tensor_engine():
    api.set_sketch_engine("tensor")
    yield
    api.set_sketch_engine("tensor")


@pytest.mark.parametrize("n,m,ncols", [(1000, 700, 1), (1000, 700, 7), (2048, 2048, 22), (333, 1500, 33),
                                       (4096, 1024, 64)])
def test_kernel_products_match_simt_and_fp64(n, m, ncols):
    g = inputs.arc_pair(n, seed=n + ncols, m=m)
    A = oo.kernel_entries(g.kernel, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, precision="mixed")
    op = api.Operator.kernel(plan)
    x = inputs.random_rhs(n, ncols, seed=1)
    xt = inputs.random_rhs(m, ncols, seed=2)
    want, want_t = A @ x, A.conj().T @ xt
    for engine, tol in (("tensor-split3", 5e-7), ("tensor-3xtf32", 2e-6), ("simt", 5e-7)):
        api.set_sketch_engine(engine)
        y = H(op.apply(T(x)))
        yt = H(op.apply(T(xt), "C"))
        assert rel(y, want) <= tol, (engine, rel(y, want))
        assert rel(yt, want_t) <= tol, (engine, rel(yt, want_t))


def test_split_k_long_sums():
    """One group with K = n = 16384 (the leaf sketches): the launch splits K
    across CTAs and adds the partial (hi, lo) sums with TwoSum."""
    n = 16384
    g = inputs.line_pair(n)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, precision="mixed")
    op = api.Operator.kernel(plan)
    x = inputs.random_rhs(n, 6, seed=5)
    rows = np.arange(0, n, 257)
    want = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt[rows], g.src) @ x
    for engine, tol in (("tensor-split3", 5e-7), ("tensor-3xtf32", 2e-6)):
        api.set_sketch_engine(engine)
        y = H(op.apply(T(x)))[rows]
        assert rel(y, want) <= tol, (engine, rel(y, want))


def test_dense_complex64_products():
    n = 1536
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, leaf=32, precision="mixed")
    op = api.Operator.dense(plan, T(A, torch.complex128))
    x = inputs.random_rhs(n, 24, seed=4)
    assert rel(H(op.apply(T(x))), A @ x) <= 2e-6
    assert rel(H(op.apply(T(x), "T")), A.T @ x) <= 2e-6


def test_mixed_factorization_on_tensor_cores_vs_oracle():
    n, eps = 2048, 1e-6
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=eps,
                    precision="mixed")
    op = api.Operator.kernel(plan)
    F = api.Factorization.factor(plan, op)
    Fo = ob.factor(oo.DenseOp(A), g.src, g.tgt, plan.L, eps, 2, 4, seed=0)
    bound = 2 * math.sqrt(plan.L + 2) * eps
    Om = ob.error_probe(n, 11, 16)
    AO = A @ Om
    assert rel(H(F.apply(T(Om, torch.complex128))), AO) <= bound
    assert np.linalg.norm(H(F.apply(T(Om, torch.complex128))) - ob.apply(Fo, Om)) <= bound * np.linalg.norm(AO)
    assert F.error(op, 16, seed=3) <= bound
