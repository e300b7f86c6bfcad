"""Full-size checks at the benchmark's configuration (2D Helmholtz line pair,
n = m = 16384, 8 points per wavelength, entries on the fly, leaf 16, tol 1e-6,
p 2, r0 16, mixed precision, the launch configuration bench.py times):

* the tensor-core sketch product (a 16384 x 16384 operator times 22 columns,
  split K across CTAs) against the oracle's FP64 kernel rows on sampled
  output rows, which the oracle computes one by one;
* the factorization's F x on sampled rows against the same exact products,
  within the error the paper bounds (Thm 5.3, with the usual factor 2);
* the sketch error of Sec. 7 (eq. error) within that bound.

The oracle appears here only as the reference of a test."""
import math

import numpy as np
import pytest
import torch

from oracle import operators as oo
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu

N, LEAF, TOL = 16384, 16, 1e-6


@pytest.fixture(scope="module")
def setup():
    g = inputs.line_pair(N)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=LEAF, tol=TOL,
                    precision="mixed", r0=16)
    op = api.Operator.kernel(plan)
    rows = np.sort(np.random.default_rng(11).choice(N, 48, replace=False))
    A_rows = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt[rows], g.src)   # FP64, 48 x 16384
    return g, plan, op, rows, A_rows


def test_sketch_product_rows_match_the_oracle(setup):
    g, plan, op, rows, A_rows = setup
    x = inputs.random_rhs(N, 22, seed=3)
    y = op.apply(api.colmajor(torch.from_numpy(x).to(torch.complex64).cuda())).cpu().numpy()
    want = A_rows @ x.astype(np.complex64).astype(np.complex128)
    # FP32-level products and FP32-level kernel entries over 16384 terms
    err = np.linalg.norm(y[rows] - want) / np.linalg.norm(want)
    assert err <= 1e-6, err


def test_factorization_rows_and_sketch_error(setup):
    g, plan, op, rows, A_rows = setup
    F = api.Factorization.factor(plan, op)
    bound = 2 * math.sqrt(plan.L + 2) * TOL
    assert F.error(op, 16, seed=7) <= bound
    x = inputs.random_rhs(N, 8, seed=5)
    y = F.apply(api.colmajor(torch.from_numpy(x).to(torch.complex64).cuda())).cpu().numpy()
    want = A_rows @ x
    err = np.linalg.norm(y[rows] - want) / np.linalg.norm(want)
    assert err <= bound, err
