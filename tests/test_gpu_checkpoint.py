"""Checkpoint files (bf_fact_save / bf_fact_load): a reloaded factorization
has the saved ranks and black-box column counts and applies bit for bit as
the saved one, in every op and both dtypes, for a mixed factorization (with
its complex64 copy) and a plain FP64 one on ragged, permuted trees; a file
for another plan, a truncated file and a file of another kind are refused."""
import os

import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_save_load_applies_bit_for_bit(tmp_path, precision):
    g = inputs.cap_pair(1500, m=1300)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, p=4,
                    precision=precision)
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    dts = (torch.complex64, torch.complex128) if precision == "mixed" else (torch.complex128,)
    xs = {}
    for dt in dts:
        xs[dt] = (api.colmajor(torch.from_numpy(inputs.random_rhs(1500, 9, seed=1)).to(dt).cuda()),
                  api.colmajor(torch.from_numpy(inputs.random_rhs(1300, 9, seed=2)).to(dt).cuda()))
    want = {(dt, op): F.apply(xs[dt][0 if op == "N" else 1], op=op).cpu().numpy() for dt in dts for op in "NTC"}
    path = tmp_path / "f.bff"
    F.save(path)
    G = api.Factorization.load(plan, path)
    for j in range(plan.lm + 1):
        assert np.array_equal(G.ranks(0, j), F.ranks(0, j))
    for j in range(plan.lm, plan.L + 1):
        assert np.array_equal(G.ranks(1, j), F.ranks(1, j))
    fi, gi = F.info(), G.info()
    assert (gi["cols_N"], gi["cols_T"], gi["stored_entries"]) == (fi["cols_N"], fi["cols_T"], fi["stored_entries"])
    for dt in dts:
        for op in "NTC":
            got = G.apply(xs[dt][0 if op == "N" else 1], op=op).cpu().numpy()
            assert np.array_equal(got, want[(dt, op)]), (dt, op)
    G.free()
    F.free()


def test_load_refuses_wrong_plan_and_bad_files(tmp_path):
    g = inputs.arc_pair(1024, seed=3)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=16, precision="mixed")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    path = tmp_path / "f.bff"
    F.save(path)
    g2 = inputs.arc_pair(2048, seed=3)
    other = api.Plan(g2.src, g2.tgt, kernel=g2.kernel, wavenumber=g2.wavenumber, leaf=16, precision="mixed")
    with pytest.raises(api.BFError):
        api.Factorization.load(other, path)
    data = path.read_bytes()
    cut = tmp_path / "cut.bff"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(api.BFError):
        api.Factorization.load(plan, cut)
    junk = tmp_path / "junk.bff"
    junk.write_bytes(b"not a factorization file" * 10)
    with pytest.raises(api.BFError):
        api.Factorization.load(plan, junk)
    with pytest.raises(api.BFError):
        api.Factorization.load(plan, tmp_path / "missing.bff")
    F.free()
