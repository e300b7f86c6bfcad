"""BF_DEBUG bounds checks: with BF_DEBUG=1 in the environment as the library
loads (or a build with -DBF_DEBUG), every stage task list of a factorization
(peeling, the centre projections) and of an apply is checked before its
launch: each output and input block inside its buffer, ranks and term counts
in range, each term's factor entries inside their block.  The same
factorizations and applies (ragged, permuted arc trees; a batch; every apply
engine) must run through the checks without an alarm and give results
identical bit for bit to a process without them."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
from paper_2002_03400_gb300 import api, inputs

out = {}
for prec, dt in (("mixed", torch.complex64), ("fp64", torch.complex128)):
    g = inputs.arc_pair(1500, seed=11)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6, precision=prec)
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.n, 37, seed=3)).to(dt).cuda())
    for eng in ("stages", "grouped", "persistent", "fused"):
        api.set_apply_engine(eng)
        for op in ("N", "C"):
            out[f"{prec}_{eng}_{op}"] = F.apply(x, op=op).cpu().numpy()
    api.set_apply_engine("auto")
    out[f"{prec}_ranks"] = np.concatenate([F.ranks(0, j) for j in range(plan.lm + 1)])
plans, ops = [], []
for i, n in enumerate((512, 1024, 777)):
    g = inputs.arc_pair(n, seed=40 + i)
    p = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=16, tol=1e-5, precision="mixed")
    plans.append(p)
    ops.append(api.Operator.kernel(p))
Fs = api.Factorization.factor_batch(plans, ops)
for i, (p, F) in enumerate(zip(plans, Fs)):
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(p.n, 4, seed=i)).to(torch.complex64).cuda())
    out[f"batch{i}"] = F.apply(x).cpu().numpy()
np.savez(sys.argv[1], **out)
"""


def _run(path, debug):
    env = dict(os.environ)
    env.pop("BF_DEBUG", None)
    if debug:
        env["BF_DEBUG"] = "1"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT, str(path)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(path)


def test_debug_checks_pass_and_change_nothing(tmp_path):
    plain = _run(tmp_path / "plain.npz", False)
    checked = _run(tmp_path / "checked.npz", True)
    assert sorted(plain.files) == sorted(checked.files)
    for k in plain.files:
        assert np.array_equal(plain[k], checked[k]), k
