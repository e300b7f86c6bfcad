"""Plan options beyond Alg. 2's defaults, through the C ABI, against the
oracle; and the failure path of the bounded device waits.

* hybrid_level (Secs. 3.3.1-3.3.3): B at any level l in [0, L-1]; l = 0 is
  the column-wise factorization, the row-wise one is l = 0 applied to A^T.
  Compared with oracle.butterfly.factor(..., hybrid_level=l): exact recovery
  of an exactly-butterfly operator with the same black-box column counts,
  and on a kernel matrix ranks +-1 and the probe gap <= 1e-6.
* accept_retries (Sec. 4.2's heuristic stop checked a posteriori by the
  sketch error of Sec. 7): with the leaf loops capped at one pass (a planted
  early stop, leaf_passes = 1) and r0 = 2, the library must retry with the
  same r0 sequence as oracle.butterfly.factor_checked and accept the same
  factorization.
* bf_debug_wait_timeout: one bounded mbarrier wait that nothing completes
  gives up after a short limit and the host reads BF_ETIMEOUT; the context
  stays usable."""
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


def rank_gap(F, Fo):
    w = 0
    for j in range(F.lm + 1):
        w = max(w, int(np.max(np.abs(F.ranks(0, j) - Fo.rV[j]))))
    for j in range(F.lm, F.L + 1):
        w = max(w, int(np.max(np.abs(F.ranks(1, j) - Fo.rU[j]))))
    return w


@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_hybrid_level_exact_recovery_and_column_counts(level):
    n, leaf, r = 1024, 16, 4
    eb = inputs.exact_butterfly(n, leaf, r, seed=1)
    Fx = api.exact_factorization(api.Plan(n=n, leaf=leaf), eb)
    bb = api.Operator.factored(Fx)
    plan = api.Plan(n=n, leaf=leaf, tol=1e-12, hybrid_level=level)
    assert plan.lm == level
    F = api.Factorization.factor(plan, bb)
    for j in range(level + 1):
        assert np.all(F.ranks(0, j) == r)
    for j in range(level, plan.L + 1):
        assert np.all(F.ranks(1, j) == r)
    Fe = ob.from_blocks(eb)
    Fo = ob.factor(oo.FactorOp(Fe), None, None, plan.L, 1e-12, 2, 4, seed=0, hybrid_level=level)
    x = inputs.random_rhs(n, 5, seed=3)
    want = ob.apply(Fe, x)
    for op in ("N", "C"):
        wop = want if op == "N" else ob.apply(Fe, x, "C")
        assert np.linalg.norm(H(F.apply(T(x), op)) - wop) <= 1e-11 * np.linalg.norm(wop)
    info = F.info()
    assert info["cols_T"] == sum(v for k, v in Fo.bb_cols.items() if k[0] in "VW")
    assert info["cols_N"] == sum(v for k, v in Fo.bb_cols.items() if k[0] in "UR")


@pytest.mark.parametrize("level", [0, 5])
def test_hybrid_level_kernel_matches_oracle(level):
    n, leaf, eps = 1024, 16, 1e-6
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=leaf, tol=eps,
                    hybrid_level=level)
    F = api.Factorization.factor(plan, api.Operator.dense(plan, T(A)))
    Fo = ob.factor(oo.DenseOp(A), g.src, g.tgt, plan.L, eps, 2, 4, seed=0, hybrid_level=level)
    assert rank_gap(F, Fo) <= 1
    Om = ob.error_probe(n, 11, 16)
    assert np.linalg.norm(H(F.apply(T(Om))) - ob.apply(Fo, Om)) <= 1e-6 * np.linalg.norm(A @ Om)


def test_hybrid_level_out_of_range_refused():
    with pytest.raises(api.BFError) as e:
        api.Plan(n=1024, leaf=16, hybrid_level=6)
    assert e.value.code == -1


def test_accept_retries_recovers_a_planted_early_stop(monkeypatch):
    n, leaf, eps = 1024, 16, 1e-6
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    L = inputs.leaf_levels(n, leaf)
    bound = 2 * math.sqrt(L + 2) * eps
    dop = oo.DenseOp(A)
    monkeypatch.setattr(ob, "leaf_loop_done", lambda r, max_rank, k, leaf_max: True)
    Fo, tried = ob.factor_checked(dop, g.src, g.tgt, L, eps, 2, 2, seed=0)
    monkeypatch.undo()
    kw = dict(kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=leaf, tol=eps, r0=2, leaf_passes=1)
    # the planted stop alone misses the bound
    p0 = api.Plan(g.src, g.tgt, **kw)
    op = api.Operator.dense(p0, T(A))
    F0 = api.Factorization.factor(p0, op)
    assert F0.error(op, 16, seed=5) > bound and F0.accept_info()["attempts"] == 1
    # with the check the library retries along the oracle's r0 sequence
    pc = api.Plan(g.src, g.tgt, accept_retries=4, **kw)
    opc = api.Operator.dense(pc, T(A))
    F = api.Factorization.factor(pc, opc)
    acc = F.accept_info()
    assert acc["attempts"] == len(tried) and acc["r0"] == tried[-1][0]
    assert acc["sketch_error"] <= bound and abs(acc["sketch_error"] - tried[-1][1]) <= 1e-6
    assert rank_gap(F, Fo) <= 1
    Om = ob.error_probe(n, 11, 16)
    assert np.linalg.norm(H(F.apply(T(Om))) - ob.apply(Fo, Om)) <= 1e-6 * np.linalg.norm(A @ Om)
    # too few retries: not converged
    pn = api.Plan(g.src, g.tgt, accept_retries=1, **kw)
    with pytest.raises(api.BFError) as e:
        api.Factorization.factor(pn, api.Operator.dense(pn, T(A)))
    assert e.value.code == -4


def test_accept_retries_accepts_a_converged_run_at_once():
    n, leaf, eps = 1024, 16, 1e-6
    g = inputs.line_pair(n)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=leaf, tol=eps,
                    precision="mixed", qr_fp64=True, accept_retries=3)
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    acc = F.accept_info()
    assert acc["attempts"] == 1 and acc["r0"] == 4 and 0 < acc["sketch_error"] <= 2 * math.sqrt(plan.L + 2) * eps


def test_bounded_wait_gives_up_and_reports_timeout():
    assert api.debug_wait_timeout(2_000_000) == -6          # 2 ms, nothing arrives: BF_ETIMEOUT
    assert api.debug_wait_timeout(0) == -1                   # limit out of range
    # the context is still usable, and the next wait is bounded at 1 s again
    n = 512
    eb = inputs.exact_butterfly(n, 16, 4, seed=2)
    F = api.exact_factorization(api.Plan(n=n, leaf=16), eb)
    x = inputs.random_rhs(n, 2, seed=1)
    assert np.linalg.norm(H(F.apply(T(x))) - ob.apply(ob.from_blocks(eb), x)) <= 1e-13 * np.linalg.norm(x) * 10
    g = inputs.line_pair(2048)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, precision="mixed")
    Fk = api.Factorization.factor(plan, api.Operator.kernel(plan))    # tensor-core kernels, bounded waits
    assert Fk.error(api.Operator.kernel(plan), 16, seed=3, dtype=torch.complex64) <= 2 * math.sqrt(plan.L + 2) * 1e-6


@pytest.mark.parametrize("case", ["line-mixed-fp64qr", "cap-ragged-mixed", "line-fp64-dense", "arc-batch"])
def test_parallel_sides_equal_sequential(case):
    """The two sides of Alg. 2 on two threads and streams (default) give the
    factorization the sequential schedule gives, bit for bit."""
    def build():
        if case == "line-mixed-fp64qr":
            g = inputs.line_pair(4096)
            p = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                         precision="mixed", r0=16, qr_fp64=True)
            return [p], [api.Operator.kernel(p)]
        if case == "cap-ragged-mixed":
            g = inputs.cap_pair(777, m=700)
            p = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, precision="mixed")
            return [p], [api.Operator.kernel(p)]
        if case == "line-fp64-dense":
            g = inputs.line_pair(1024)
            A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
            p = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6)
            return [p], [api.Operator.dense(p, T(A))]
        plans, ops = [], []
        for i, n in enumerate((1024, 2048, 1024, 4096)):
            g = inputs.arc_pair(n, seed=40 + i)
            p = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=1e-5,
                         precision="mixed", seed=i, qr_fp64=True)
            plans.append(p)
            ops.append(api.Operator.kernel(p))
        return plans, ops

    plans, ops = build()
    out = {}
    for on in (True, False):
        api.set_parallel_sides(on)
        if len(plans) == 1:
            out[on] = [api.Factorization.factor(plans[0], ops[0])]
        else:
            out[on] = api.Factorization.factor_batch(plans, ops)
    api.set_parallel_sides(True)
    for Fp, Fs, p in zip(out[True], out[False], plans):
        for j in range(p.lm + 1):
            assert np.array_equal(Fp.ranks(0, j), Fs.ranks(0, j))
        for j in range(p.lm, p.L + 1):
            assert np.array_equal(Fp.ranks(1, j), Fs.ranks(1, j))
        x = T(inputs.random_rhs(p.n, 3, seed=7), torch.complex128)
        assert torch.equal(Fp.apply(x), Fs.apply(x))
        assert Fp.info()["cols_N"] == Fs.info()["cols_N"] and Fp.info()["cols_T"] == Fs.info()["cols_T"]
