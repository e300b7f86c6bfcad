"""Persistent apply (bf_set_apply_engine 3: all stages of eq.
hybrid_butterfly_mat in one cooperative launch, each output block started
once the blocks it reads are written) and grouped apply (engine 4: runs of
1-4 stages per launch, each run's inner stages in shared memory, one CTA per
connected group of blocks).  Per block both form the same FMA chains as the
stage launches (terms in order, k ascending), so F x, F^T x and F^H x must
equal the stage engine's bit for bit:
* ragged, permuted 2-D trees (arc pair, leaf 24: blocks of every rank, odd
  row offsets) and a 3-D pair of adjacent hemispheres, whose ranks exceed
  one round of staged rows (K > 48) and one block of rows (M > 16);
* column counts of one column, partial and whole 64-column slices and
  more than one slice, in complex64 and complex128;
* x and y the same buffer (in place): the persistent engine steps aside
  (its stages overlap), the grouped engine's first run reads x before its
  last run writes y;
* the tuner choosing among the engines keeps every result."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _reset_engine():
    yield
    api.set_apply_engine("auto")
    api.set_grouped_depth(0)
    api.set_grouped_merge(0)


_CACHE = {}


def _factor(case, dtype):
    if (case, dtype) not in _CACHE:
        _CACHE[(case, dtype)] = _build(case, dtype)
    return _CACHE[(case, dtype)]


def _engine(name):
    if name.startswith("grouped"):
        api.set_apply_engine("grouped")
        api.set_grouped_depth(int(name.split("-")[1]))
    else:
        api.set_apply_engine(name)


def _build(case, dtype):
    prec = "mixed" if dtype == torch.complex64 else "fp64"
    if case == "arc":
        g = inputs.arc_pair(1500, seed=11)
        plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, precision=prec)
    else:
        g = inputs.hemisphere_pair(4096)
        plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=32, tol=1e-4, p=4, r0=32,
                        precision=prec)
    return plan, api.Factorization.factor(plan, api.Operator.kernel(plan))


@pytest.mark.parametrize("engine", ["persistent", "grouped-1", "grouped-2", "grouped-3", "grouped-4"])
@pytest.mark.parametrize("case", ["arc", "hemi"])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_engine_equals_stage_apply(engine, case, dtype):
    plan, F = _factor(case, dtype)
    if case == "hemi":
        assert max(int(F.ranks(0, j).max()) for j in range(plan.lm + 1)) > 16
    for nrhs in (1, 3, 37, 64, 130):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.n, nrhs, seed=nrhs)).to(dtype).cuda())
        xm = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.m, nrhs, seed=nrhs + 7)).to(dtype).cuda())
        api.set_apply_engine("stages")
        ref = {"N": F.apply(x), "T": F.apply(xm, op="T"), "C": F.apply(xm, op="C")}
        _engine(engine)
        got = {"N": F.apply(x), "T": F.apply(xm, op="T"), "C": F.apply(xm, op="C")}
        for op in ("N", "T", "C"):
            assert torch.equal(got[op], ref[op]), (engine, case, nrhs, op)


@pytest.mark.parametrize("merge", [1, 2, 4, 8])
@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_group_merging_keeps_results(merge, depth, dtype):
    """Independent groups merged into one CTA (up to 1, 2, 4, 8 blocks of a
    run's last stage) change which CTA computes a block, never its FMA
    chain: grouped and persistent applies equal the stage launches bit for
    bit on the ragged arc tree, 1 to 130 columns (slices of 32 columns and
    more take the column-major staging of x and y)."""
    plan, F = _factor("arc", dtype)
    api.set_grouped_merge(merge)
    api.set_grouped_depth(depth)
    for nrhs in (1, 37, 64, 130):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.n, nrhs, seed=nrhs + 1)).to(dtype).cuda())
        xm = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.m, nrhs, seed=nrhs + 9)).to(dtype).cuda())
        api.set_apply_engine("stages")
        ref = {"N": F.apply(x), "C": F.apply(xm, op="C")}
        for eng in ("grouped", "persistent"):
            api.set_apply_engine(eng)
            got = {"N": F.apply(x), "C": F.apply(xm, op="C")}
            for op in ("N", "C"):
                assert torch.equal(got[op], ref[op]), (eng, merge, depth, nrhs, op)


def test_group_merging_knob_range():
    with pytest.raises(api.BFError):
        api.set_grouped_merge(-1)
    with pytest.raises(api.BFError):
        api.set_grouped_merge(17)


@pytest.mark.parametrize("engine", ["persistent", "grouped-3"])
def test_in_place_apply(engine):
    g = inputs.line_pair(2048)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                    precision="mixed")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(2048, 8, seed=2)).to(torch.complex64).cuda())
    api.set_apply_engine("stages")
    ref = F.apply(x)
    _engine(engine)
    xy = x.clone(memory_format=torch.preserve_format)
    F.apply_into(xy, xy)
    torch.cuda.synchronize()
    assert torch.equal(xy, ref)


def test_tuner_with_persistent_engine_keeps_results():
    plan, F = _factor("arc", torch.complex64)
    for nrhs in (1, 64):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.n, nrhs, seed=4)).to(torch.complex64).cuda())
        before = F.apply(x)
        ms = F.tune(nrhs, torch.complex64)
        assert ms > 0
        assert torch.equal(F.apply(x), before)
    with pytest.raises(KeyError):
        api.set_apply_engine("bogus")
    with pytest.raises(api.BFError):
        api.check(api.lib().bf_set_apply_engine(5))
    with pytest.raises(api.BFError):
        api.set_grouped_depth(5)
