"""The 3D experiment's geometry on the GPU (Sec. 7.3, Table 2): two unit
hemispheres that touch along the equator, exp(i k r)/(4 pi r) at 10 points
per wavelength, the paper's 3-D parameters p = 4, r0 = 64, tol 1e-6 (weak
admissibility: every level keeps blocks whose point sets touch, so ranks
grow with n).  Through the C ABI against the FP64 oracle on the same seeded
points: ranks within +-1 per block, the probe gap (Sec. 7, eq. error
columns) within 1e-6 of ||A Omega|| in FP64 and within the mixed path's
3-D tolerance 2e-6 (tests/test_oracle_precision.py) in mixed precision,
the sketch error within the Thm 5.3 bound, and the centre-level ranks
above those of two separated caps at the same sampling."""
import math

import numpy as np
import pytest
import torch

from oracle import butterfly as ob
from oracle import operators as oo
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def T(x, dtype=torch.complex128):
    return api.colmajor(torch.from_numpy(np.asarray(x)).to(dtype).cuda())


def H(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def hemi1024():
    n, eps = 1024, 1e-6
    g = inputs.hemisphere_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_3D, g.wavenumber, g.tgt, g.src)
    L = inputs.leaf_levels(n, 16)
    Fo = ob.factor(oo.DenseOp(A), g.src, g.tgt, L, eps, 4, 64, seed=0)
    return g, A, Fo


@pytest.mark.parametrize("precision,qr_fp64,gap_tol", [("fp64", False, 1e-6), ("mixed", True, 2e-6),
                                                       ("mixed", False, 2e-6)])
def test_hemispheres_match_oracle(hemi1024, precision, qr_fp64, gap_tol):
    g, A, Fo = hemi1024
    n, eps = 1024, 1e-6
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz3d", wavenumber=g.wavenumber, leaf=16, tol=eps, p=4, r0=64,
                    precision=precision, qr_fp64=qr_fp64)
    op = api.Operator.kernel(plan)
    F = api.Factorization.factor(plan, op)
    pS, _, pT, _ = plan.trees()
    assert np.array_equal(pS, Fo.permS) and np.array_equal(pT, Fo.permT)
    worst = 0
    for j in range(plan.lm + 1):
        worst = max(worst, int(np.max(np.abs(F.ranks(0, j) - Fo.rV[j]))))
    for j in range(plan.lm, plan.L + 1):
        worst = max(worst, int(np.max(np.abs(F.ranks(1, j) - Fo.rU[j]))))
    assert worst <= 1
    Om = ob.error_probe(n, 11, 16)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    gap = np.linalg.norm(H(F.apply(T(Om, dt))) - ob.apply(Fo, Om)) / np.linalg.norm(A @ Om)
    assert gap <= gap_tol, gap
    assert F.error(op, 16, seed=5, dtype=dt) <= 2 * math.sqrt(plan.L + 2) * eps


def test_hemisphere_ranks_exceed_separated_caps():
    """Weak admissibility on the GPU: centre-level ranks of the touching
    hemispheres above those of separated caps at the same sampling, and
    growing from n = 2048 to 8192."""
    mid = {}
    for n in (2048, 8192):
        for name, g in (("hemi", inputs.hemisphere_pair(n)), ("caps", inputs.cap_pair(n, ppw=10.0))):
            plan = api.Plan(g.src, g.tgt, kernel="helmholtz3d", wavenumber=g.wavenumber, leaf=16, tol=1e-6, p=4,
                            r0=64, precision="mixed", qr_fp64=True)
            op = api.Operator.kernel(plan)
            F = api.Factorization.factor(plan, op)
            assert F.error(op, 16, seed=3, dtype=torch.complex64) <= 2 * math.sqrt(plan.L + 2) * 1e-6
            mid[name, n] = int(F.ranks(0, plan.lm).max())
    assert mid["hemi", 2048] > mid["caps", 2048] and mid["hemi", 8192] > mid["caps", 8192]
    assert mid["hemi", 8192] > mid["hemi", 2048]
