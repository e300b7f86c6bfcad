"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Several results are correct at once (bases are unique only up to a unitary
rotation), so factors are never compared entry by entry: the tests compare
ranks (within +-1 per block), applies of the factorization to probe columns,
the sketch error of Sec. 7 and the black-box column schedule.  Tolerances:
FP64 path -- products agree with the oracle to 1e-6 of ||A Omega|| (the
target; ~1e-13 when every rank agrees), sketch errors within the Thm 5.3
bound 2*sqrt(L+2)*eps; mixed path -- the same bounds (its FP32 products
carry ~1e-7 relative error, below eps = 1e-6)."""
import math

import numpy as np
import pytest
import torch

from oracle import butterfly as ob
from oracle import operators as oo
from oracle import rng as orng
from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def T(x, dtype=torch.complex128):
    return torch.from_numpy(np.asarray(x)).to(dtype).cuda()


def H(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def bound(L, eps):
    return 2 * math.sqrt(L + 2) * eps


def ranks_close(F, Fo, tol=1):
    worst = 0
    for j in range(F.lm + 1):
        worst = max(worst, int(np.max(np.abs(F.ranks(0, j) - Fo.rV[j]))))
    for j in range(F.lm, F.L + 1):
        worst = max(worst, int(np.max(np.abs(F.ranks(1, j) - Fo.rU[j]))))
    assert worst <= tol, f"rank difference {worst}"
    return worst


def probe_gap(F, Fo, A_apply, n, cols=16, dtype=torch.complex128):
    Om = ob.error_probe(n, 11, cols)
    yg = H(F.apply(T(Om, dtype)))
    yo = ob.apply(Fo, Om)
    return np.linalg.norm(yg - yo) / np.linalg.norm(A_apply(Om))


# --------------------------------------------------------------------------- RNG

@pytest.mark.parametrize("seed,sid,row0,rows,c0,c1", [(0, 1 << 8, 0, 1000, 0, 7),
                                                      (12345678901, (4 << 8) | 3, 3, 501, 5, 9),
                                                      (7, 5 << 8, 0, 1, 0, 16)])
def test_gaussian_matches_oracle(seed, sid, row0, rows, c0, c1):
    o = orng.gaussian(seed, sid, np.arange(row0, row0 + rows), c0, c1)
    g = H(api.gaussian(seed, sid, rows, c0, c1, row0=row0))
    assert np.max(np.abs(g - o)) <= 1e-13 * np.abs(o).max()
    g32 = H(api.gaussian(seed, sid, rows, c0, c1, dtype=torch.complex64, row0=row0))
    assert np.max(np.abs(g32 - o)) <= 1e-6 * np.abs(o).max()


# ------------------------------------------------------------------------- apply

@pytest.mark.parametrize("n,leaf,r", [(2048, 32, 8), (512, 8, 4), (1024, 16, 6)])
def test_apply_exact_butterfly(n, leaf, r):
    eb = inputs.exact_butterfly(n, leaf, r, seed=1)
    plan = api.Plan(n=n, leaf=leaf)
    F = api.exact_factorization(plan, eb)
    Fo = ob.from_blocks(eb)
    for nrhs in (1, 5, 33, 100):
        x = inputs.random_rhs(n, nrhs, seed=nrhs)
        for op in ("N", "T", "C"):
            yo = ob.apply(Fo, x, op)
            yg = H(F.apply(T(x), op))
            assert np.linalg.norm(yg - yo) <= 1e-13 * np.linalg.norm(yo)
            y32 = H(F.apply(T(x, torch.complex64), op))
            assert np.linalg.norm(y32 - yo) <= 1e-5 * np.linalg.norm(yo)


@pytest.mark.parametrize("engine", ["stages", "grouped-1", "grouped-2", "grouped-3", "grouped-4", "persistent",
                                    "fused"])
def test_every_apply_engine_matches_oracle(engine):
    """Each apply engine against the oracle's apply of the same exact
    butterfly (eq. hybrid_butterfly_mat), every op, both dtypes."""
    n, leaf, r = 1024, 16, 6
    eb = inputs.exact_butterfly(n, leaf, r, seed=4)
    F = api.exact_factorization(api.Plan(n=n, leaf=leaf), eb)
    Fo = ob.from_blocks(eb)
    if engine.startswith("grouped"):
        api.set_apply_engine("grouped")
        api.set_grouped_depth(int(engine.split("-")[1]))
    else:
        api.set_apply_engine(engine)
    try:
        for nrhs in (1, 33, 70):
            x = inputs.random_rhs(n, nrhs, seed=nrhs + 3)
            for op in ("N", "T", "C"):
                yo = ob.apply(Fo, x, op)
                assert np.linalg.norm(H(F.apply(T(x), op)) - yo) <= 1e-13 * np.linalg.norm(yo), (engine, op)
                y32 = H(F.apply(T(x, torch.complex64), op))
                assert np.linalg.norm(y32 - yo) <= 1e-5 * np.linalg.norm(yo), (engine, op)
    finally:
        api.set_apply_engine("auto")
        api.set_grouped_depth(0)


def test_apply_strided_and_empty():
    n = 512
    eb = inputs.exact_butterfly(n, 16, 4, seed=2)
    plan = api.Plan(n=n, leaf=16)
    F = api.exact_factorization(plan, eb)
    Fo = ob.from_blocks(eb)
    x = inputs.random_rhs(n, 3, seed=3)
    big = torch.zeros((3, n + 40), dtype=torch.complex128, device="cuda").t()    # ld = n + 40
    big[:n] = T(x)
    yg = H(F.apply(big[:n]))
    assert np.allclose(yg, ob.apply(Fo, x), atol=1e-12)
    out = F.apply(torch.zeros((n, 0), dtype=torch.complex128, device="cuda"))
    assert out.shape == (n, 0)


# ------------------------------------------------------------------- factorization

def _dense_case(n, leaf, eps, precision, geom="line", seed=0, qr_fp64=False):
    g = {"line": lambda: inputs.line_pair(n), "arc": lambda: inputs.arc_pair(n, seed=5),
         "cap": lambda: inputs.cap_pair(n)}[geom]()
    kern = oo.HELMHOLTZ_3D if geom == "cap" else oo.HELMHOLTZ_2D
    A = oo.kernel_entries(kern, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, kernel=int(kern), wavenumber=g.wavenumber, leaf=leaf, tol=eps,
                    precision=precision, seed=seed, qr_fp64=qr_fp64)
    return g, A, plan


@pytest.mark.parametrize("precision,qr_fp64", [("fp64", False), ("mixed", False), ("mixed", True)])
def test_factor_dense_line_matches_oracle(precision, qr_fp64):
    """Plain FP64 method on the 1024-point parallel-lines workload; the mixed
    path with its float-float QR (default) and with the FP64 QR."""
    n, leaf, eps = 1024, 16, 1e-6
    g, A, plan = _dense_case(n, leaf, eps, precision, qr_fp64=qr_fp64)
    pS, offS, pT, offT = plan.trees()
    op = api.Operator.dense(plan, T(A))
    F = api.Factorization.factor(plan, op)
    dop = oo.DenseOp(A)
    Fo = ob.factor(dop, g.src, g.tgt, plan.L, eps, 2, 4, seed=0)
    assert np.array_equal(pS, Fo.permS) and np.array_equal(pT, Fo.permT)
    worst = ranks_close(F, Fo)
    gap = probe_gap(F, Fo, lambda X: A @ X, n)
    assert gap <= 1e-6
    if precision == "fp64" and worst == 0:
        assert gap <= 1e-12
        info = F.info()
        assert info["cols_T"] == sum(v for k, v in Fo.bb_cols.items() if k[0] in "VW")
        assert info["cols_N"] == sum(v for k, v in Fo.bb_cols.items() if k[0] in "UR")
    e = F.error(op, 16, seed=5)
    eo = ob.sketch_error(dop, Fo, seed=5)
    assert e <= bound(plan.L, eps) and abs(e - eo) <= 1e-6


def test_mixed_qr_float_float_vs_fp64():
    """The mixed path's float-float QR and its FP64 QR reveal the same ranks
    (up to +-1 at the threshold) and the same sketch-error level."""
    n, leaf, eps = 4096, 16, 1e-6
    g = inputs.line_pair(n)
    out = {}
    for q in (False, True):
        plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=leaf, tol=eps,
                        precision="mixed", r0=16, qr_fp64=q)
        op = api.Operator.kernel(plan)
        F = api.Factorization.factor(plan, op)
        out[q] = (F, F.error(op, 16, seed=3, dtype=torch.complex64), plan)
    (Ff, ef, plan), (Fd, ed, _) = out[False], out[True]
    worst = 0
    for j in range(plan.lm + 1):
        worst = max(worst, int(np.max(np.abs(Ff.ranks(0, j) - Fd.ranks(0, j)))))
    for j in range(plan.lm, plan.L + 1):
        worst = max(worst, int(np.max(np.abs(Ff.ranks(1, j) - Fd.ranks(1, j)))))
    assert worst <= 1
    assert ef <= bound(plan.L, eps) and ed <= bound(plan.L, eps)
    assert abs(ef - ed) <= 0.1 * bound(plan.L, eps)


@pytest.mark.parametrize("geom,n,m,leaf", [("arc", 1000, 900, 16), ("cap", 777, 700, 24), ("line", 300, 300, 8)])
def test_factor_ragged_and_permuted(geom, n, m, leaf):
    """Ragged trees (n not leaf * 2^L, m != n) and non-identity permutations."""
    eps = 1e-6
    g = {"arc": lambda: inputs.arc_pair(n, seed=2, m=m), "cap": lambda: inputs.cap_pair(n, m=m),
         "line": lambda: inputs.line_pair(n, m)}[geom]()
    A = oo.kernel_entries(g.kernel, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=leaf, tol=eps)
    op = api.Operator.kernel(plan)
    F = api.Factorization.factor(plan, op)
    Fo = ob.factor(oo.DenseOp(A), g.src, g.tgt, plan.L, eps, 2, 4, seed=0)
    ranks_close(F, Fo)
    assert probe_gap(F, Fo, lambda X: A @ X, n) <= 1e-6
    x = inputs.random_rhs(m, 3, seed=4)
    for opn in ("T", "C"):
        yo = ob.apply(Fo, x, opn)
        assert np.linalg.norm(H(F.apply(T(x), opn)) - yo) <= 1e-6 * np.linalg.norm(yo)


def test_kernel_operator_equals_dense_operator():
    n, leaf, eps = 1024, 16, 1e-6
    g, A, plan = _dense_case(n, leaf, eps, "fp64")
    Fd = api.Factorization.factor(plan, api.Operator.dense(plan, T(A)))
    Fk = api.Factorization.factor(plan, api.Operator.kernel(plan))
    x = inputs.random_rhs(n, 4, seed=9)
    yd, yk = H(Fd.apply(T(x))), H(Fk.apply(T(x)))
    assert np.linalg.norm(yd - yk) <= 1e-6 * np.linalg.norm(yd)
    opk = api.Operator.kernel(plan)
    assert np.allclose(H(opk.apply(T(x))), A @ x, rtol=1e-12, atol=1e-12 * np.abs(A @ x).max())


@pytest.mark.parametrize("n,leaf,r", [(2048, 32, 8), (1024, 8, 4)])
def test_exact_recovery(n, leaf, r):
    """Sec. 7.1: recovery of an exactly-butterfly operator to 1e-11."""
    eb = inputs.exact_butterfly(n, leaf, r, seed=1)
    src_plan = api.Plan(n=n, leaf=leaf)
    Fx = api.exact_factorization(src_plan, eb)
    bb = api.Operator.factored(Fx)
    plan = api.Plan(n=n, leaf=leaf, tol=1e-12)
    F = api.Factorization.factor(plan, bb)
    for j in range(plan.lm + 1):
        assert np.all(F.ranks(0, j) == r)
    for j in range(plan.lm, plan.L + 1):
        assert np.all(F.ranks(1, j) == r)
    assert F.error(bb, 16, seed=3) <= 1e-11
    Fo = ob.from_blocks(eb)
    assert probe_gap(F, Fo, lambda X: ob.apply(Fo, X), n) <= 1e-11


def test_callback_black_box_and_failures():
    n, leaf, r = 512, 16, 4
    eb = inputs.exact_butterfly(n, leaf, r, seed=4)
    Fx = api.exact_factorization(api.Plan(n=n, leaf=leaf), eb)
    L = api.lib()
    calls = {"n": 0}

    def fn(op, ncols, X, ldx, Y, ldy, dtype, stream):
        calls["n"] += 1
        if op == 0:
            return L.bf_apply(Fx._h, ncols, X, ldx, Y, ldy, dtype, stream)
        return L.bf_apply_T(Fx._h, 1, ncols, X, ldx, Y, ldy, dtype, stream)

    cb = api.Operator.callback(n, n, fn)
    plan = api.Plan(n=n, leaf=leaf, tol=1e-12)
    F = api.Factorization.factor(plan, cb)
    assert calls["n"] > 0
    assert F.error(cb, 16, seed=1) <= 1e-11

    bad = api.Operator.callback(n, n, lambda *a: 7)
    with pytest.raises(api.BFError) as e:
        api.Factorization.factor(plan, bad)
    assert e.value.code == -3
    tight = api.Plan(n=n, leaf=leaf, tol=1e-12, r_max=4, r0=2)
    with pytest.raises(api.BFError) as e:
        api.Factorization.factor(tight, api.Operator.factored(Fx))
    assert e.value.code == -4
    with pytest.raises(api.BFError) as e:                 # the plan alone needs ~10 KB
        api.Plan(n=n, leaf=leaf, tol=1e-12, mem_cap=4096)
    assert e.value.code == -2
    capped = api.Plan(n=n, leaf=leaf, tol=1e-12, mem_cap=64 * 1024)
    with pytest.raises(api.BFError) as e:                 # the first two sketch buffers need ~98 KB
        api.Factorization.factor(capped, api.Operator.factored(Fx))
    assert e.value.code == -2


def test_composition_black_box():
    """A = A1 A2 given only through the factors of A1 and A2 (Sec. 1,
    category (ii)); recompression recovers the product."""
    n, leaf = 1024, 16
    g = inputs.line_pair(n)
    A1 = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)     # rows tgt, cols src
    A2 = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.src, g.tgt)     # rows src, cols tgt
    p1 = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=leaf, tol=1e-9)
    F1 = api.Factorization.factor(p1, api.Operator.dense(p1, T(A1)))
    p2 = api.Plan(g.tgt, g.src, leaf=leaf, tol=1e-9)
    F2 = api.Factorization.factor(p2, api.Operator.dense(p2, T(A2)))
    comp = api.Operator.composed(api.Operator.factored(F1), api.Operator.factored(F2))
    plan = api.Plan(g.tgt, g.tgt, leaf=leaf, tol=1e-6)
    F = api.Factorization.factor(plan, comp)
    x = inputs.random_rhs(n, 4, seed=8)
    want = A1 @ (A2 @ x)
    assert np.linalg.norm(H(F.apply(T(x))) - want) <= bound(plan.L, 1e-6) * np.linalg.norm(want) * 2


def test_dft_against_numpy_fft():
    n = 2048
    g = inputs.dft_points(n)
    plan = api.Plan(g.src, g.tgt, kernel="dft", leaf=16, tol=1e-9)
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    x = inputs.random_rhs(n, 3, seed=2)
    want = np.fft.fft(x, axis=0)
    assert np.linalg.norm(H(F.apply(T(x))) - want) <= bound(plan.L, 1e-9) * np.linalg.norm(want) * 3
